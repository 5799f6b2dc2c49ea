"""dg_rhs_noalloc: the FP64 right-hand side for callers that cannot allocate device
memory (a framework's memory pool, an allocator that forbids raw cudaMalloc after
start-up, or a process that already holds all device memory).  Its scratch is a fixed
file-scope device array, so these tests check that its output matches dg_rhs (the
context-based entry point) on two calls in a row -- the second call must not be
affected by what the first left in the shared array -- and that a problem too large
for the array is refused before any GPU work.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W


def _entry():
    import paper_2306_05002_gb300 as pkg
    lib = pkg.load()
    f = lib.dg_rhs_noalloc
    f.argtypes = [ctypes.POINTER(pkg.dg_mesh), ctypes.c_int, ctypes.POINTER(pkg.dg_eos), ctypes.c_double,
                  ctypes.c_double, ctypes.POINTER(pkg.dg_opts), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return pkg, f


def _structs(pkg, wl):
    kw = wl.problem_kwargs()
    p, Gamma, eps = kw.pop("p"), kw.pop("Gamma"), kw.pop("eps")
    m, e, o = pkg.make_structs(**kw)
    return m, p, e, Gamma, eps, o


@pytest.mark.gpu
def test_noalloc_matches_dg_rhs_on_two_calls_in_a_row(dg):
    import torch
    pkg, f = _entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two different problems back to back: the second call sees the first one's leftovers
    for wl in (W.drop_2d(n=16, p=3, seed=2), W.drop_2d(n=11, p=4, seed=7)):
        m, p, e, Gamma, eps, o = _structs(pkg, wl)
        w = torch.from_numpy(wl.w.copy()).cuda()
        L = torch.full_like(w, float("nan"))
        st = f(ctypes.byref(m), p, ctypes.byref(e), Gamma, eps, ctypes.byref(o),
               ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(L.data_ptr()), stream)
        assert st == 0
        solver = pkg.Solver(wl)
        ref = solver.dg_rhs(w)
        torch.cuda.synchronize()
        got, ref = L.cpu().numpy(), ref.cpu().numpy()
        solver.close()
        for v in range(7):
            scale = max(np.abs(ref[v]).max(), 1e-300)
            assert np.abs(got[v] - ref[v]).max() <= 1e-12 * scale, v


def test_noalloc_rejects_problems_larger_than_its_scratch():
    """Checked before any GPU work, so this runs without a GPU too."""
    pkg, f = _entry()
    wl = W.Workload(name="big", dim=2, nx=256, ny=256, p=3)
    m, p, e, Gamma, eps, o = _structs(pkg, wl)
    st = f(ctypes.byref(m), p, ctypes.byref(e), 1.0, 0.01, ctypes.byref(o),
           ctypes.c_void_p(16), ctypes.c_void_p(32), None)
    assert st == -1  # DG_ERR_ARG
