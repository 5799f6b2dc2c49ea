"""GPU checks of the kinematic mode (Sec. 4.1): phase field and level set advected by a
prescribed velocity with classical RK4, FP64, against the oracle.

* one right-hand side: max_n |L - L_orc| <= 1e-12 max_n S per field (S: the oracle's sum of
  absolute contributions), p = 1..5, uniform and Rider-Kothe velocities, at several times;
* RK4 steps (one graph of 8 steps plus single steps) against the oracle's RK4: no pressure
  recovery here, so the states agree to 1e-12 of their scale plus the step count times the
  per-stage bound;
* the Rider-Kothe vortex over a full period on the 16 x 16, p = 3 mesh (64^2 degrees of
  freedom, as in the paper's table): the drop comes back, its phase-field mass is kept to
  1e-8, and the L1 error sits near the paper's p = 3 value (a results-level comparison, not
  a parity pin: the paper does not state Gamma and eps for this test).
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _kin(orc, wl):
    return orc.Problem(**wl.problem_kwargs()), orc.Velocity(**wl.velocity_kwargs())


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("vel", ["uniform", "rider_kothe"])
def test_kin_rhs_parity(orc, dg, p, vel):
    import torch
    wl = W.rider_kothe(n=5, p=p)
    if vel == "uniform":
        wl.vel, wl.u0, wl.v0 = "uniform", 0.8, -0.35
    rng = np.random.default_rng(p)
    w = wl.w + 0.05 * rng.uniform(-1, 1, wl.w.shape)    # broken, discontinuous state
    pb, vc = _kin(orc, wl)
    s = dg.KinematicSolver(wl)
    for t in (0.0, 0.7, 1.9):
        L_ref, S = orc.kin_rhs(pb, vc, t, w, want_scale=True)
        L = s.dg_kin_rhs(torch.from_numpy(w.copy()).cuda(), t).cpu().numpy()
        for v in range(2):
            assert np.abs(L[v] - L_ref[v]).max() <= 1e-12 * S[v].max(), (t, v)
    assert s.dg_status_read() == 0
    s.close()


@pytest.mark.parametrize("nsteps", [3, 11])
def test_kin_rk4_parity(orc, dg, nsteps):
    import torch
    wl = W.rider_kothe(n=8, p=3, T=0.5)
    pb, vc = _kin(orc, wl)
    t0, dt = 0.05, 2e-4
    ref = orc.kin_rk4(pb, vc, wl.w, t0, dt, nsteps)
    _, S = orc.kin_rhs(pb, vc, t0, wl.w, want_scale=True)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_kin_step(w, t0, dt, nsteps)
    got = w.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    for v in range(2):
        bound = 1e-12 * np.abs(ref[v]).max() + 4 * nsteps * 1e-12 * dt * S[v].max()
        assert np.abs(got[v] - ref[v]).max() <= bound, v


def test_kin_step_t0_is_read_at_run_time(dg):
    """The captured graph reads the start time from device memory: stepping from t0 in two calls
    equals one call, and a different t0 changes the result of a time-dependent velocity."""
    import torch
    wl = W.rider_kothe(n=6, p=2, T=1.0)
    s = dg.KinematicSolver(wl)
    a = torch.from_numpy(wl.w.copy()).cuda()
    b = a.clone()
    c = a.clone()
    dt = 1e-4
    s.dg_kin_step(a, 0.1, dt, 10)
    s.dg_kin_step(b, 0.1, dt, 4)
    s.dg_kin_step(b, 0.1 + 4 * dt, dt, 6)
    s.dg_kin_step(c, 0.3, dt, 10)
    s.close()
    assert torch.allclose(a, b, rtol=0, atol=1e-13)
    assert (a - c).abs().max().item() > 1e-9


def _rider_kothe(dg, orc, n):
    import torch
    wl = W.rider_kothe(n=n, p=3)
    xi, wt = orc.gll(wl.p)
    M = np.tile(np.outer(wt, wt).ravel() * 0.25 * wl.hx * wl.hy, wl.nx * wl.ny)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    half = wl.nsteps // 2
    s.dg_kin_step(w, 0.0, wl.dt, half)
    w_half = w.cpu().numpy()
    s.dg_kin_step(w, half * wl.dt, wl.dt, wl.nsteps - half)
    w_end = w.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    l1_half = np.sum(M * np.abs(w_half[0] - wl.w[0]))
    l1_end = np.sum(M * np.abs(w_end[0] - wl.w[0]))
    mass_err = abs(np.sum(M * (w_end[0] - wl.w[0])) / np.sum(M * wl.w[0]))
    return l1_half, l1_end, mass_err


def test_rider_kothe_full_period(orc, dg):
    """16 x 16, 32 x 32 and 64 x 64, p = 3 (the paper's 64^2, 128^2 and 256^2 DoF rows), vortex
    centred on the domain, eps = 0.75 of the node spacing: the stretched drop comes back (the
    error at T is well below the one at T/2), the L1 error falls under refinement, sits within a
    factor 2 of the paper's p = 3 values at 128^2 and 256^2 (4.83e-3, 1.23e-3) and below its 64^2
    value (1.75e-2) -- results-level, since the paper states neither Gamma nor eps for this
    test -- and the phase-field mass is conserved to round-off (the nodal velocity is the
    discrete curl of the stream function, see the oracle pins)."""
    res = {n: _rider_kothe(dg, orc, n) for n in (16, 32, 64)}
    for n in (16, 32, 64):
        l1_half, l1_end, mass_err = res[n]
        assert l1_end < 0.5 * l1_half, (n, res)
    assert res[16][1] < 1.75e-2, res
    for n, paper in ((32, 4.83e-3), (64, 1.23e-3)):
        assert 0.5 * paper < res[n][1] < 2 * paper, (n, res)
    assert res[64][1] < res[32][1] < res[16][1], res
    for n in (16, 32, 64):
        assert res[n][2] < 1e-12, res



def _droplet_l1(dg, orc, n, p, eps):
    import torch
    wl = W.kin_drop(n=n, p=p, eps=eps)
    xi, wt = orc.gll(wl.p)
    M = np.tile(np.outer(wt, wt).ravel() * 0.25 * wl.hx * wl.hy, wl.nx * wl.ny)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_kin_step(w, 0.0, wl.dt, wl.nsteps)  # one period: the exact solution is the initial one
    out = w.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    return float(np.sum(M * np.abs(out[0] - wl.w[0])))


def test_droplet_advection_convergence(orc, dg):
    """The linear advection of a droplet (Sec. 4.1: R = 0.15, u = (1, 0), one period).  With the
    paper's eps = 0.05 the L1 error falls under refinement for p = 1, 2, 3 and with p at a fixed
    mesh, but the level set's cone tip at the drop centre, where phi (1 - phi) is still 0.045
    (the drop is 3 eps in radius) and the discrete normal is O(1) wrong within an element, adds
    an O(h^2) error; with eps = 0.02 (phi (1 - phi) = 5.5e-4 there) p = 3 converges at the optimal
    rate p + 1."""
    paper = {(p, n): _droplet_l1(dg, orc, n, p, 0.05) for p in (1, 2, 3) for n in (10, 20, 40)}
    for p in (1, 2, 3):
        assert paper[(p, 40)] < paper[(p, 20)] < paper[(p, 10)], paper
    for n in (10, 20, 40):
        assert paper[(3, n)] < paper[(2, n)] < paper[(1, n)], paper
    thin = [_droplet_l1(dg, orc, n, 3, 0.02) for n in (20, 40, 80)]
    rates = [np.log2(a / b) for a, b in zip(thin, thin[1:])]
    assert min(rates) > 3.5, (thin, rates)


@pytest.mark.parametrize("elem", ["quad", "tri"])
def test_kin_step_size_changes_between_calls(dg, elem):
    """The captured kinematic step graphs read dt (and the start time) from device memory: calls
    with changing step sizes on one context give exactly what fresh contexts give, on rectangles
    and triangles, single steps and 8-step graphs alike."""
    import torch
    wl = W.rider_kothe(n=8, p=3, elem=elem)
    plan = [(wl.dt, 3), (0.5 * wl.dt, 9), (wl.dt, 1), (0.25 * wl.dt, 8)]
    s = dg.KinematicSolver(wl)
    a = torch.from_numpy(wl.w.copy()).cuda()
    t = 0.0
    for dt, n in plan:
        s.dg_kin_step(a, t, dt, n)
        t += n * dt
    s.close()
    b = torch.from_numpy(wl.w.copy()).cuda()
    t = 0.0
    for dt, n in plan:
        f = dg.KinematicSolver(wl)
        f.dg_kin_step(b, t, dt, n)
        f.close()
        t += n * dt
    assert torch.equal(a, b)
