"""Batched ensemble (FP32-bulk): every problem of a mixed-order batch against the FP64 oracle
(one and several SSP-RK3 steps: relative L2 error of every variable and of the pressure within
1e-6, as the single-problem FP32-bulk path is held), and, problem by problem, against what the
single-problem FP32-bulk path computes.  Both run the same kernel bodies, but the compiler may
fuse multiply-adds differently in the two kernels, so they agree to FP32 rounding: 16 eps32 per
stage relative to max|w| (one step: ~1 ulp observed; nine steps: ~23 ulps)."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem

pytestmark = pytest.mark.gpu


TOL_STAGE = 16 * 2.0 ** -23


def _single(dg, wl, nsteps):
    import torch
    s = dg.Solver(wl, precision="fp32bulk")
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, nsteps)
    out = d.cpu().numpy()
    s.close()
    return out


def _l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("nsteps,orders", [(1, (2, 3, 4, 5)), (4, (2, 3, 4, 5)), (3, (1,))])
def test_batch_matches_oracle(orc, dg, nsteps, orders):
    """Each problem of a batch of orders 2..5, or of order 1 (meshes of 4 to 9 elements a side,
    drops and bubbles) after `nsteps` batched steps against the oracle's SSP-RK3 steps of the same
    problem: relative L2 error of every stored variable and of the pressure <= 1e-6."""
    import torch
    wls = W.ensemble(n=8, seed=11, nmin=4, nmax=9, orders=orders)
    assert {wl.p for wl in wls} == set(orders)
    bs = dg.BatchSolver(wls)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], nsteps)
    torch.cuda.synchronize()
    bs.close()
    for wl, st in zip(wls, states):
        pb = problem(orc, wl)
        ref = orc.rk3(pb, wl.w, wl.dt, nsteps)
        got = st.cpu().numpy()
        for v in (0, 1, 2, 3, 4, 5, 6):
            assert _l2(got[v], ref[v]) <= 1e-6, (wl.name, v, _l2(got[v], ref[v]))
        P_got, P_ref = orc.primitives(pb, got)[3], orc.primitives(pb, ref)[3]
        assert _l2(P_got, P_ref) <= 1e-6, (wl.name, _l2(P_got, P_ref))


@pytest.mark.parametrize("nsteps", [1, 3])
def test_batch_with_walls_pressure_top_and_gravity_matches_oracle(orc, dg, nsteps):
    """A batch whose problems have walls and gravity (inviscid): the paper's Rayleigh-Taylor domain
    (slip sides, no-slip bottom, the pressure top), a no-slip box with a perturbed interface, and a
    periodic drop (g = 0), against the oracle's SSP-RK3: phi, psi, m_l, rho E and P within 1e-6
    (relative L2) as above, the momenta within the FP32 storage bound of the pressure gradient."""
    import torch
    a = W.rayleigh_taylor_paper(nx=4, ny=12, p=4)
    b = W.rayleigh_taylor(n=6, p=3, seed=5)
    for wl in (a, b):
        wl.viscous = wl.surface_tension = False
        wl.gravity = True
    c = W.drop_2d(n=6, p=2, seed=3)
    wls = [a, b, c]
    bs = dg.BatchSolver(wls)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], nsteps)
    torch.cuda.synchronize()
    bs.close()
    for wl, st in zip(wls, states):
        pb = problem(orc, wl)
        ref = orc.rk3(pb, wl.w, wl.dt, nsteps)
        got = st.cpu().numpy()
        for v in (0, 1, 2, 3, 6):
            assert _l2(got[v], ref[v]) <= 1e-6, (wl.name, v, _l2(got[v], ref[v]))
        # the momenta of fluids at rest under gravity: what moves them is the hydrostatic imbalance, so
        # the FP32 storage error of P (4 eps32 max|P|) through the pressure gradient, (2/h) max_i
        # sum_c |D_ic| per stage, bounds the difference (the bound of the multi-step FP32-bulk test)
        xi, _ = orc.gll(wl.p)
        D = orc.lagrange_deriv(wl.p, xi)
        h = min(wl.hx, wl.hy)
        P_max = np.abs(orc.primitives(pb, ref)[3]).max()
        extra = 3 * nsteps * wl.dt * 4 * np.finfo(np.float32).eps * P_max * (2.0 / h) * np.abs(D).sum(axis=1).max()
        for v in (4, 5):
            tol = 1e-6 * np.abs(ref[v]).max() + extra
            assert np.abs(got[v] - ref[v]).max() <= tol, (wl.name, v, np.abs(got[v] - ref[v]).max(), tol)
        P_got, P_ref = orc.primitives(pb, got)[3], orc.primitives(pb, ref)[3]
        assert _l2(P_got, P_ref) <= 1e-6, (wl.name, _l2(P_got, P_ref))


@pytest.mark.parametrize("nsteps", [1, 9])
def test_batch_equals_single_problem_runs(dg, nsteps):
    import torch
    wls = W.ensemble(n=7, seed=4, nmin=3, nmax=12, orders=(1, 2, 3, 4, 5))
    bs = dg.BatchSolver(wls)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], nsteps)
    torch.cuda.synchronize()
    for wl, st in zip(wls, states):
        ref = _single(dg, wl, nsteps)
        got = st.cpu().numpy()
        for v in range(7):
            scale = max(np.abs(ref[v]).max(), 1e-300)
            assert np.abs(got[v] - ref[v]).max() <= TOL_STAGE * 3 * nsteps * scale, (wl.name, v)
    bs.close()


def test_batch_new_pointers_and_steps_are_picked_up(dg):
    """A second call with other state tensors and other step sizes (descriptor re-upload,
    same captured graph)."""
    import torch
    wls = W.ensemble(n=3, seed=5, nmin=4, nmax=8, orders=(2, 3))
    bs = dg.BatchSolver(wls)
    a = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(a, [wl.dt for wl in wls], 1)
    b = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(b, [0.5 * wl.dt for wl in wls], 2)
    torch.cuda.synchronize()
    def close(got, ref, nsteps):
        scale = np.abs(ref).max(axis=1, keepdims=True)
        return np.all(np.abs(got - ref) <= TOL_STAGE * 3 * nsteps * scale)
    for wl, x, y in zip(wls, a, b):
        assert close(x.cpu().numpy(), _single(dg, wl, 1), 1)
        wl2 = W.Workload(**{k: getattr(wl, k) for k in wl.problem_kwargs()}, name=wl.name)
        wl2.w, wl2.dt = wl.w, 0.5 * wl.dt
        assert close(y.cpu().numpy(), _single(dg, wl2, 2), 2)
    bs.close()


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
def test_every_tile_variant_matches_single_problem_runs(dg, tile):
    """Each compiled tile (elements per block x register budget) gives the single-problem result."""
    import torch
    wls = W.ensemble(n=5, seed=6, nmin=3, nmax=10, orders=(1, 2, 3, 4, 5))
    bs = dg.BatchSolver(wls, tile=tile)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], 2)
    torch.cuda.synchronize()
    tiles = bs.dg_batch_tiles()
    assert sorted(t["p"] for t in tiles) == sorted({wl.p for wl in wls})
    for wl, st in zip(wls, states):
        ref = _single(dg, wl, 2)
        got = st.cpu().numpy()
        for v in range(7):
            scale = max(np.abs(ref[v]).max(), 1e-300)
            assert np.abs(got[v] - ref[v]).max() <= TOL_STAGE * 6 * scale, (wl.name, v)
    bs.close()


def test_tuner_reports_a_tile_per_order(dg):
    import torch
    wls = W.ensemble(n=6, seed=7, nmin=8, nmax=24, orders=(2, 3, 4, 5))
    bs = dg.BatchSolver(wls)
    assert bs.dg_batch_tiles() == []          # nothing tuned before the first step
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], 1)
    tiles = bs.dg_batch_tiles()
    assert sorted(t["p"] for t in tiles) == sorted({wl.p for wl in wls})
    for t in tiles:
        assert t["epb"] >= 1 and t["minb"] >= 1 and 0 < t["ms"] <= t["ms_default_tile"]
    bs.close()


def test_full_ensemble_sampled_problems_match_single_runs(dg):
    """The 256-problem ensemble the benchmark times (seed 4, 35.2M nodes, tuned tiles): after two
    batched steps every state is finite, and eight problems spread over the four orders agree
    with their single-problem FP32-bulk runs to the stage tolerance."""
    import torch
    wls = W.ensemble(n=256, seed=4)
    bs = dg.BatchSolver(wls)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], 2)
    torch.cuda.synchronize()
    assert all(bool(torch.isfinite(st).all()) for st in states)
    picks = []
    for p in (2, 3, 4, 5):
        idx = [k for k, wl in enumerate(wls) if wl.p == p]
        picks += [idx[0], idx[-1]]
    for k in picks:
        ref = _single(dg, wls[k], 2)
        got = states[k].cpu().numpy()
        for v in range(7):
            scale = max(np.abs(ref[v]).max(), 1e-300)
            assert np.abs(got[v] - ref[v]).max() <= TOL_STAGE * 3 * 2 * scale, (wls[k].name, v)
    bs.close()


def test_order5_ensemble_problems_stay_finite(dg):
    """The order-5 bubbles among the ensemble's first 13 problems (seed 4), 300 steps at their own
    step size, batched and one by one in FP64 and FP32-bulk: finite, and no status raised.  (At
    the acoustic limit that suits p <= 4 these problems overflow within 200 steps in either
    precision; order 5 takes 0.9 of it.)"""
    import torch
    wls = [wl for wl in W.ensemble(n=13, seed=4) if wl.p == 5 and wl.nx <= 60]
    assert len(wls) >= 2
    for prec in ("fp64", "fp32bulk"):
        for wl in wls:
            s = dg.Solver(wl, precision=prec)
            d = torch.from_numpy(wl.w.copy()).cuda()
            s.dg_step(d, wl.dt, 300)
            assert bool(torch.isfinite(d).all()), (prec, wl.name)
            assert s.dg_status_read() == 0, (prec, wl.name)
            s.close()
    bs = dg.BatchSolver(wls)
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    bs.dg_batch_step(states, [wl.dt for wl in wls], 300)
    torch.cuda.synchronize()
    assert all(bool(torch.isfinite(st).all()) for st in states)
    bs.close()
