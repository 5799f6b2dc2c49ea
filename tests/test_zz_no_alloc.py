"""dg_rhs_noalloc: the FP64 right-hand side for callers that cannot allocate device memory (a
framework's memory pool, an allocator that forbids raw cudaMalloc after start-up, or a process
that already holds all device memory).  Its scratch is a fixed file-scope device array shared by
every call, so these tests check that its output matches dg_rhs (the context-based entry point)
on calls in a row -- each call must not be affected by what the one before left in the shared
array -- over every kernel family it reaches (orders 1 to 5, 1D and 2D, viscous stress, gravity,
surface tension, walls, the pressure boundary, lifted gradients), and that a problem too large for the array, or
one it does not cover, is refused before any GPU work.

This file is collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
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


CASES = {
    "drop_16x16_p3": lambda: W.drop_2d(n=16, p=3, seed=2),
    "drop_11x11_p4": lambda: W.drop_2d(n=11, p=4, seed=7),
    "drop_9x9_p1": lambda: W.drop_2d(n=9, p=1, seed=3),
    "bubble_6x6_p5": lambda: W.drop_2d(n=6, p=5, seed=4, water_inside=False),
    "slab_1d_p3": lambda: W.slab_1d(nx=37, p=3),
    # the Rayleigh-Taylor set-up: viscous stress, gravity, surface tension, no-slip walls
    "rayleigh_taylor_8x8_p4": lambda: W.rayleigh_taylor(n=8, p=4, seed=3),
    # the paper's Rayleigh-Taylor domain: slip sides, no-slip bottom, pressure top
    "rt_paper_4x12_p4": lambda: W.rayleigh_taylor_paper(nx=4, ny=12, p=4),
    # BR1-lifted gradients on a state that jumps at every face
    "drop_lifted_8x8_p3": lambda: _jumping(W.drop_2d(n=8, p=3, seed=5), lift=True),
}


def _jumping(wl, lift):
    """The workload with its phase field and level set perturbed node by node (seeded)."""
    rng = np.random.default_rng(9)
    w = np.array(wl.w)
    w[0] = np.clip(w[0] + 0.05 * rng.uniform(-1, 1, wl.N), 0.0, 1.0)
    w[1] = w[1] + 0.05 * rng.uniform(-1, 1, wl.N)
    wl.w = W.conserved(wl, w[0], w[1], 1e5, 1.0, 0.5)
    wl.grad_lift = lift
    return wl


def _noalloc_vs_rhs(pkg, f, wl, stream):
    import torch
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
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * scale, (wl.name, v)


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_dg_rhs_twice(dg, case):
    """The same problem twice in a row: the second call runs on the first one's leftovers."""
    import torch
    pkg, f = _entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    wl = CASES[case]()
    for _ in range(2):
        _noalloc_vs_rhs(pkg, f, wl, stream)


@pytest.mark.gpu
def test_noalloc_matches_dg_rhs_on_two_calls_in_a_row(dg):
    """Different problems back to back (a large one, then smaller ones with other kernel
    families and scratch layouts, then the first again)."""
    import torch
    pkg, f = _entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for case in ("drop_16x16_p3", "rayleigh_taylor_8x8_p4", "slab_1d_p3", "drop_11x11_p4", "drop_16x16_p3"):
        _noalloc_vs_rhs(pkg, f, CASES[case](), stream)


def test_noalloc_rejects_problems_larger_than_its_scratch():
    """Checked before any GPU work, so this runs without a GPU too."""
    pkg, f = _entry()
    wl = W.Workload(name="big", dim=2, nx=256, ny=256, p=3)
    m, p, e, Gamma, eps, o = _structs(pkg, wl)
    st = f(ctypes.byref(m), p, ctypes.byref(e), 1.0, 0.01, ctypes.byref(o),
           ctypes.c_void_p(16), ctypes.c_void_p(32), None)
    assert st == -1  # DG_ERR_ARG


def test_noalloc_rejects_what_it_does_not_cover():
    """Before any GPU work: FP32-bulk (DG_ERR_UNSUPPORTED), triangles (DG_ERR_UNSUPPORTED), an
    order beyond 5 (DG_ERR_UNSUPPORTED), unpaired periodic sides and aliased arrays (DG_ERR_ARG)."""
    pkg, f = _entry()
    wl = W.drop_2d(n=4, p=3, seed=2)
    args = lambda m, p, e, o, w=16, L=32: (ctypes.byref(m), p, ctypes.byref(e), 1.0, 0.01, ctypes.byref(o),
                                          ctypes.c_void_p(w), ctypes.c_void_p(L), None)
    m, p, e, _, _, o = _structs(pkg, wl)
    o.prec = 1
    assert f(*args(m, p, e, o)) == -7
    m, p, e, _, _, o = _structs(pkg, wl)
    m.elem = 1
    assert f(*args(m, p, e, o)) == -7
    m, p, e, _, _, o = _structs(pkg, wl)
    assert f(*args(m, 6, e, o)) == -7
    m.bc[0] = 1
    assert f(*args(m, p, e, o)) == -1
    m, p, e, _, _, o = _structs(pkg, wl)
    assert f(*args(m, p, e, o, w=16, L=16)) == -1
