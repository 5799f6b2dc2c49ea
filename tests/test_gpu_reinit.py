"""GPU checks of the level-set re-initialisation (end of Sec. 3) against the oracle: psi after
0 and several pseudo-time iterations, for full-model contexts (FP64 and FP32-bulk, 1D and 2D,
periodic and walls) and kinematic contexts; every other field of the state is left untouched.
No pressure recovery is involved, so the states agree to 1e-12 of the scale of psi per
iteration."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem

pytestmark = pytest.mark.gpu


def _defaults(wl):
    h = min(wl.hx, wl.hy) if wl.dim == 2 else wl.hx
    q = 2 * wl.p + 1
    nu = h / (2 * (wl.p + 1))
    return nu, min(0.5 * h / q, 0.1 * h * h / (q * q * nu))


@pytest.mark.parametrize("make,precision", [
    (lambda: W.drop_2d(n=8, p=3, seed=2), "fp64"),
    (lambda: W.drop_2d(n=6, p=4, seed=3), "fp32bulk"),
    (lambda: W.slab_1d(nx=30, p=3), "fp64"),
    (lambda: W.rayleigh_taylor(n=6, p=2, seed=3), "fp64"),      # no-slip walls
])
@pytest.mark.parametrize("niter", [0, 7])
def test_reinit_full_model_context(orc, dg, make, precision, niter):
    import torch
    wl = make()
    nu, dtau = _defaults(wl)
    s = dg.Solver(wl, precision=precision)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_reinit(w, niter)                       # library defaults for nu and dtau
    got = w.cpu().numpy()
    s.close()
    pb = problem(orc, wl)
    ref = orc.reinit(pb, wl.w[0], niter, nu, dtau)
    assert np.array_equal(np.delete(got, 1, axis=0), np.delete(wl.w, 1, axis=0))
    scale = np.abs(ref).max()
    assert np.abs(got[1] - ref).max() <= 1e-12 * scale * (1 + niter), np.abs(got[1] - ref).max() / scale


def test_reinit_kinematic_context(orc, dg):
    import torch
    wl = W.rider_kothe(n=8, p=3)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    nu, dtau = 0.01, 2e-4
    s.dg_reinit(w, 5, nu, dtau)
    got = w.cpu().numpy()
    s.close()
    ref = orc.reinit(orc.Problem(**wl.problem_kwargs()), wl.w[0], 5, nu, dtau)
    assert np.array_equal(got[0], wl.w[0])
    assert np.abs(got[1] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_reinit_relaxes_gradient_on_the_gpu(orc, dg):
    """200 iterations on a 16 x 16, p = 3 drop: |grad psi| near the interface (from the oracle's
    broken gradient of the GPU result) moves from ~1/(4 eps) towards 1."""
    import torch
    wl = W.drop_2d(n=16, p=3, seed=2)
    s = dg.Solver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_reinit(w, 0)
    g0 = w[1].cpu().numpy()
    s.dg_reinit(w, 200)
    g1 = w[1].cpu().numpy()
    s.close()
    pb = problem(orc, wl)
    band = np.abs(wl.w[1]) < wl.eps
    def dev(psi):
        return np.abs(orc.reinit_rhs(pb, -np.ones(wl.N), psi, 0.0)[band]).max()   # | |grad psi| - 1 |
    assert dev(g1) < 0.25 * dev(g0), (dev(g0), dev(g1))
