"""The OpenMP build of the oracle (used only to time it on all host cores) computes exactly what
the plain, pinned build computes: its parallel loops are over elements or nodes whose iterations
write only their own entries, so every sum keeps its order."""
import subprocess

import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W


@pytest.fixture(scope="module")
def omp(orc):
    try:
        orc.build(openmp=True)
    except (subprocess.CalledProcessError, OSError) as exc:   # a compiler without OpenMP
        pytest.skip(f"no OpenMP build: {exc}")
    return orc


@pytest.mark.parametrize("make", [
    lambda: W.drop_2d(n=8, p=3, seed=2),
    lambda: W.rayleigh_taylor(n=6, p=4, seed=3),
    lambda: W.rayleigh_taylor_paper(nx=3, ny=12, p=3),
])
def test_openmp_build_is_bitwise_identical(omp, make):
    wl = make()
    pb = omp.Problem(**wl.problem_kwargs())
    rng = np.random.default_rng(0)
    w = wl.w * (1.0 + 1e-3 * rng.standard_normal(wl.w.shape))
    assert np.array_equal(omp.rhs_threads(pb, w, 4), omp.rhs(pb, w))
    assert np.array_equal(omp.rk3(pb, wl.w, wl.dt, 2, threads=3), omp.rk3(pb, wl.w, wl.dt, 2))
