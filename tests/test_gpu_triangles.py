"""GPU checks of the kinematic mode on triangles (the paper's mesh (b), Sec. 4.1), FP64, against
the oracle:

* one right-hand side: max_n |L - L_orc| <= 1e-12 max_n S per field (S: the oracle's sum of
  absolute contributions), p = 1..4, uniform and Rider-Kothe velocities, at several times, on a
  mesh whose triangle count leaves a ragged last group, and on one large enough that every CTA
  of the persistent grid walks several groups;
* RK4 steps (a graph of 8 steps plus single steps) against the oracle's RK4;
* the Rider-Kothe vortex over a full period on 16 x 16 and 32 x 32 cells, p = 3: the drop comes
  back, its mass is kept to round-off, and the L1 error falls under refinement, matches the
  rectangles' and sits near the paper's mesh (b) p = 3 values (a results-level comparison: the
  paper states neither Gamma nor eps).
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _kin(orc, wl):
    return orc.Problem(**wl.problem_kwargs()), orc.Velocity(**wl.velocity_kwargs())


def _broken(wl, seed):
    rng = np.random.default_rng(seed)
    return wl.w + 0.05 * rng.uniform(-1, 1, wl.w.shape)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("vel", ["uniform", "rider_kothe"])
def test_tri_rhs_parity(orc, dg, p, vel):
    import torch
    wl = W.rider_kothe(n=5, p=p, elem="tri")
    wl.ny, wl.y1 = 3, wl.y0 + 3 * wl.hx              # 5 x 3 cells, 30 triangles: a ragged last group
    wl.w = W.rider_kothe(n=5, p=p, elem="tri").w[:, :wl.N]
    if vel == "uniform":
        wl.vel, wl.u0, wl.v0 = "uniform", 0.8, -0.35
    w = _broken(wl, p)
    pb, vc = _kin(orc, wl)
    s = dg.KinematicSolver(wl)
    for t in (0.0, 0.7, 1.9):
        L_ref, S = orc.tri_rhs(pb, vc, t, w, want_scale=True)
        L = s.dg_kin_rhs(torch.from_numpy(w.copy()).cuda(), t).cpu().numpy()
        for v in range(2):
            assert np.abs(L[v] - L_ref[v]).max() <= 1e-12 * S[v].max(), (t, v)
    assert s.dg_status_read() == 0
    s.close()


def test_tri_rhs_parity_many_groups_per_cta(orc, dg):
    import torch
    wl = W.rider_kothe(n=96, p=3, elem="tri")          # 18432 triangles, 2304 groups of 8
    w = _broken(wl, 11)
    pb, vc = _kin(orc, wl)
    s = dg.KinematicSolver(wl)
    L_ref, S = orc.tri_rhs(pb, vc, 0.3, w, want_scale=True)
    L = s.dg_kin_rhs(torch.from_numpy(w.copy()).cuda(), 0.3).cpu().numpy()
    s.close()
    for v in range(2):
        assert np.abs(L[v] - L_ref[v]).max() <= 1e-12 * S[v].max(), v


@pytest.mark.parametrize("nsteps", [3, 11])
def test_tri_rk4_parity(orc, dg, nsteps):
    import torch
    wl = W.rider_kothe(n=8, p=3, T=0.5, elem="tri")
    pb, vc = _kin(orc, wl)
    t0, dt = 0.05, 1e-4
    ref = orc.tri_rk4(pb, vc, wl.w, t0, dt, nsteps)
    _, S = orc.tri_rhs(pb, vc, t0, wl.w, want_scale=True)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_kin_step(w, t0, dt, nsteps)
    got = w.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    for v in range(2):
        bound = 1e-12 * np.abs(ref[v]).max() + 4 * nsteps * 1e-12 * dt * S[v].max()
        assert np.abs(got[v] - ref[v]).max() <= bound, v


def test_tri_reinit_is_rejected(dg):
    import torch
    wl = W.rider_kothe(n=4, p=2, elem="tri")
    s = dg.KinematicSolver(wl)
    with pytest.raises(dg.DGError):
        s.dg_reinit(torch.from_numpy(wl.w.copy()).cuda(), 5)
    s.close()


def _rider_kothe(dg, orc, n, elem, p=3):
    import torch
    wl = W.rider_kothe(n=n, p=p, elem=elem)
    pb = orc.Problem(**wl.problem_kwargs())
    if elem == "tri":
        integral = lambda f: orc.tri_integral(pb, f)
    else:
        _, wt = orc.gll(wl.p)
        M = np.tile(np.outer(wt, wt).ravel() * 0.25 * wl.hx * wl.hy, wl.nx * wl.ny)
        integral = lambda f: float(np.sum(M * f))
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    half = wl.nsteps // 2
    s.dg_kin_step(w, 0.0, wl.dt, half)
    w_half = w.cpu().numpy()
    s.dg_kin_step(w, half * wl.dt, wl.dt, wl.nsteps - half)
    w_end = w.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    l1_half = integral(np.abs(w_half[0] - wl.w[0]))
    l1_end = integral(np.abs(w_end[0] - wl.w[0]))
    mass_err = abs(integral(w_end[0] - wl.w[0]) / integral(wl.w[0]))
    return l1_half, l1_end, mass_err


def test_rider_kothe_orders_and_meshes_against_the_paper(orc, dg):
    """The paper's L1 table (results level: the paper states neither Gamma nor eps; here
    eps = 0.75 of the node spacing, Gamma = 1).  p = 3 on 16^2, 32^2 and 64^2 cells (64^2, 128^2,
    256^2 DoF) and p = 1 on 32^2 and 128^2 cells (64^2 and 256^2 DoF), on triangles (mesh (b)) and
    rectangles (mesh (a)): the p = 3 errors fall under refinement, sit within a factor 2 of the
    paper's p = 3 rows at 128^2 and 256^2 and below them at 64^2; p = 3 beats p = 1 at matched DoF,
    as the paper reports; the two meshes give nearly the same interface (the paper's finding);
    and the triangles keep the phase-field mass to round-off (the paper: 1e-10 down to machine
    precision for p = 3; the velocity is exact at the quadrature points)."""
    paper_p3 = {"quad": (1.75e-2, 4.83e-3, 1.23e-3), "tri": (1.58e-2, 4.03e-3, 1.18e-3)}
    p3 = {m: [_rider_kothe(dg, orc, n, m, p=3) for n in (16, 32, 64)] for m in ("tri", "quad")}
    p1 = {m: [_rider_kothe(dg, orc, n, m, p=1) for n in (32, 128)] for m in ("tri", "quad")}
    for m in ("tri", "quad"):
        l1 = [r[1] for r in p3[m]]
        assert all(r[1] < 0.5 * r[0] for r in p3[m]), (m, p3[m])
        assert l1[2] < l1[1] < l1[0], (m, l1)
        assert l1[0] < paper_p3[m][0], (m, l1)
        for got, paper in zip(l1[1:], paper_p3[m][1:]):
            assert 0.5 * paper < got < 2 * paper, (m, l1)
        assert l1[0] < p1[m][0][1] and l1[2] < p1[m][1][1], (m, l1, p1[m])
    for k in range(3):
        assert 0.67 < p3["tri"][k][1] / p3["quad"][k][1] < 1.5, (k, p3)
        assert p3["tri"][k][2] < 1e-10, (k, p3["tri"])
