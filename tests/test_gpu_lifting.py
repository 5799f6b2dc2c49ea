"""GPU parity of the BR1-lifted gradient option (dg_opts.grad_lift = 1) against the oracle with the
same option, on states whose phase field and level set jump at every face (where the lifting acts):
one right-hand side at 1e-12 of the oracle's scale S for orders 1..5, 1D and 2D, walls, the
pressure boundary and the viscous, gravity and surface-tension terms; a few SSP-RK3 steps; and
the contexts that do not build lifted gradients refuse the option."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem
from tests.test_gpu_parity import _assert_parity, _broken

pytestmark = pytest.mark.gpu


def _lifted(wl, seed=4):
    """The option on, and the state perturbed node by node (in 1D only phi and psi: the 1D state
    keeps rho v = 0)."""
    wl.grad_lift = True
    if wl.dim == 2:
        wl.w = np.array(_broken(wl, seed=seed))
    else:
        rng = np.random.default_rng(seed)
        phi = np.clip(wl.w[0] + 0.05 * rng.uniform(-1, 1, wl.N), 0.0, 1.0)
        psi = wl.w[1] + 0.05 * rng.uniform(-1, 1, wl.N)
        wl.w = np.array(W.conserved(wl, phi, psi, 1e5, 1.0, 0.0))
    return wl


def _rhs(orc, dg, wl):
    import torch
    L_ref, S = orc.rhs(problem(orc, wl), wl.w, want_scale=True)
    s = dg.Solver(wl)
    L = s.dg_rhs(torch.from_numpy(wl.w.copy()).cuda()).cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    return L, L_ref, S


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_lifted_rhs_drop(orc, dg, p):
    _assert_parity(*_rhs(orc, dg, _lifted(W.drop_2d(n=6, p=p, seed=2))))


@pytest.mark.parametrize("p", [2, 4])
def test_lifted_rhs_slab_1d(orc, dg, p):
    _assert_parity(*_rhs(orc, dg, _lifted(W.slab_1d(nx=23, p=p))))


def test_lifted_rhs_walls_viscous_surface_tension(orc, dg):
    wl = W.rayleigh_taylor(n=6, p=4, seed=3)
    wl.bc = ("slip", "slip", "noslip", "slip")
    _assert_parity(*_rhs(orc, dg, _lifted(wl)))


def test_lifted_rhs_pressure_boundary(orc, dg):
    _assert_parity(*_rhs(orc, dg, _lifted(W.rayleigh_taylor_paper(nx=4, ny=12, p=3))))


def test_lifting_changes_the_rhs(orc, dg):
    """The option is in effect: on a discontinuous state the lifted and broken right-hand sides of
    the phase field differ far beyond rounding (on the GPU as in the oracle)."""
    import torch
    wl = _lifted(W.drop_2d(n=6, p=3, seed=2))
    s1 = dg.Solver(wl)
    L1 = s1.dg_rhs(torch.from_numpy(wl.w.copy()).cuda()).cpu().numpy()
    s1.close()
    wl.grad_lift = False
    s0 = dg.Solver(wl)
    L0 = s0.dg_rhs(torch.from_numpy(wl.w.copy()).cuda()).cpu().numpy()
    s0.close()
    _, S = orc.rhs(problem(orc, wl), wl.w, want_scale=True)
    assert np.abs(L1[0] - L0[0]).max() > 1e-6 * S[0].max()


def test_lifted_steps_against_oracle(orc, dg):
    import torch
    wl = _lifted(W.drop_2d(n=8, p=3, seed=5))
    s = dg.Solver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(w, wl.dt, 5)
    got = w.cpu().numpy()
    s.close()
    ref = orc.rk3(problem(orc, wl), wl.w, wl.dt, 5)
    for v in range(7):
        sc = np.abs(ref[v]).max()
        assert np.abs(got[v] - ref[v]).max() <= 5 * 3 * 4 * 2.0 ** -52 * 5e4 * sc, v


def test_contexts_without_lifted_gradients_refuse_the_option(dg):
    import torch
    wl = W.drop_2d(n=4, p=3, seed=2)
    wl.grad_lift = True
    with pytest.raises(dg.DGError) as ex:
        dg.Solver(wl, precision="fp32bulk")
    assert ex.value.status == -7
    with pytest.raises(dg.DGError) as ex:
        dg.BatchSolver([wl])
    assert ex.value.status == -7
    s = dg.Solver(wl)  # FP64: built, but without a discrete adjoint
    w = torch.from_numpy(wl.w.copy()).cuda()
    with pytest.raises(dg.DGError) as ex:
        s.dg_rhs_vjp(w, w.clone())
    assert ex.value.status == -7
    s.close()
