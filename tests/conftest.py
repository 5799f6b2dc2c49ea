import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def dg():
    """The product library (built in-tree); GPU tests only."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2306_05002_gb300 as pkg
    pkg.load()  # raises if the extension is missing
    return pkg


@pytest.fixture(autouse=True)
def _bounds_checked_build(request):
    """Under DGPF_CHECKED=1 (the GPU tests run on the bounds-checked library, see
    tests/test_gpu_checked.py): every GPU test must run on that library and leave the count of
    bounds failures where it found it.  A no-op otherwise."""
    if os.environ.get("DGPF_CHECKED") != "1" or request.node.get_closest_marker("gpu") is None:
        yield
        return
    import gc

    import paper_2306_05002_gb300 as pkg
    checked, before = pkg.check_build()
    assert checked, "DGPF_CHECKED=1 but the loaded library is not the bounds-checked build"
    yield
    gc.collect()  # contexts a test dropped are destroyed here, and bits they still hold counted
    _, after = pkg.check_build()
    assert after == before, f"{after - before} bounds failure(s) in the bounds-checked build"
