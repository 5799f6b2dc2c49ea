"""The bounds-checked build (libdgpf_check.so: the library's sources with -DDG_CHECK, where every
global access of the two-phase model's kernels checks its index against its array and a failed
check is latched and the access skipped), the stand-in for a memory checker on this GPU pool.

* its self-test: an inconsistent node count planted on the device (no access leaves its
  allocation) is caught;
* the GPU suites (FP64, FP32-bulk, batched, walls and normals, lifted gradients, checkpoints, the
  adjoint, the kinematic mode on rectangles and triangles, the re-initialisation, the
  allocation-free entry) run again in a child process on the checked library, each test also
  required to leave the process's count of bounds failures unchanged (tests/conftest.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_fp32bulk.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_walls_normals.py", "tests/test_gpu_lifting.py", "tests/test_checkpoint.py",
          "tests/test_gpu_adjoint.py", "tests/test_gpu_kinematic.py", "tests/test_gpu_triangles.py",
          "tests/test_gpu_reinit.py", "tests/test_zz_no_alloc.py"]


def _checked_lib_path():
    import paper_2306_05002_gb300 as pkg
    return pkg.LIB_CHECK_PATH


def test_checked_build_selftest(dg):
    if not os.path.exists(_checked_lib_path()):
        pytest.fail("libdgpf_check.so is missing: __graft_entry__.build() builds it")
    code = ("import ctypes, paper_2306_05002_gb300 as pkg, torch; torch.cuda.init(); lib = pkg.load(); "
            "print(pkg.check_build()[0], lib.dg_check_selftest(None), pkg.check_build()[1])")
    env = dict(os.environ, DGPF_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split() == ["True", "1", "0"], r.stdout
    # the normal build has no checks
    assert dg.load().dg_check_selftest(None) == -7 and dg.check_build() == (False, 0)


def test_gpu_suites_on_the_checked_build(dg):
    env = dict(os.environ, DGPF_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    import re
    m = re.search(r"(\d+) passed", r.stdout)
    # the suites hold 195 GPU tests: all of them ran, none failed or was skipped
    assert m and int(m.group(1)) >= 190 and " failed" not in r.stdout and " skipped" not in r.stdout, r.stdout[-2000:]
