"""GPU checks of the FP32-bulk path (FP32 stage arithmetic on the reduced energy
rho E - Cmix(phi), FP64 only where the pressure is recovered).

* one right-hand side against the FP64 oracle: max_n |L - L_orc| <= 2e-6 max_n S_v per
  variable (S: the oracle's scale of the cancelling terms; FP32 has 6e-8 unit round-off
  and a node sees a few tens of contributions), plus, for phi and psi, the FP32 storage
  error of the field carried through the transport derivative (see _storage_bound);
* a full 500-step run of the 64 x 64, p = 3 drop against the FP64 path: relative L2
  error of phi and P <= 1e-5 (the accuracy target of this mode), u within 1e-3;
* interface equilibrium: a uniform-(u, P) drop keeps P within 1e-5 relative.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem

pytestmark = pytest.mark.gpu
TOL32 = 2e-6


def _storage_bound(orc, wl, w):
    """FP32 storage error of the state carried through the right-hand side (S does not contain
    it: S holds the magnitudes of the terms, not of the stored fields):
    * phi and psi through the transport derivative u.grad(f):
      4 eps32 max|f| max|u| (2/h) max_i sum_c |D_ic|;
    * the Lax-Friedrichs dissipation of each conserved field q (the FP32 internal state: m_l,
      rho u, and the reduced energy rho E - Cmix(phi)) at a face: 4 eps32 lambda_max max|q|
      max(M^-1 w_f), which matters where the jumps, and with them S, vanish (a boundary state
      equal to the interior one)."""
    xi, wt = orc.gll(wl.p)
    D = orc.lagrange_deriv(wl.p, xi)
    prim = orc.primitives(problem(orc, wl), w)
    umax = np.max(np.hypot(prim[1], prim[2]))
    h = min(wl.hx, wl.hy)
    e32 = np.finfo(np.float32).eps
    g = 4 * e32 * umax * (2.0 / h) * np.abs(D).sum(axis=1).max()
    out = {0: g * np.abs(w[0]).max(), 1: g * np.abs(w[1]).max()}
    lam = np.max(np.hypot(prim[1], prim[2]) + prim[4])
    minv_f = 1.0 / (wt[-1] * 0.5 * h)
    C = [wl.gamma[l] * wl.pinf[l] / (wl.gamma[l] - 1) for l in range(2)]
    Cmix = w[0] * C[0] + (1 - w[0]) * C[1]
    stored = {2: w[2], 3: w[3], 4: w[4], 5: w[5], 6: w[6] - Cmix}
    for v, q in stored.items():
        out[v] = 4 * e32 * lam * np.abs(q).max() * minv_f
    return out


def _rhs32(orc, dg, wl, w=None):
    import torch
    w = wl.w if w is None else w
    L_ref, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    s = dg.Solver(wl, precision="fp32bulk")
    L = s.dg_rhs(torch.from_numpy(np.array(w)).cuda()).cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    extra = _storage_bound(orc, wl, w)
    for v in range(7):
        sc = S[v].max()
        if sc == 0:
            continue
        err = np.abs(L[v] - L_ref[v]).max()
        assert err <= TOL32 * sc + extra.get(v, 0.0), (v, err / sc, extra.get(v, 0.0) / sc)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_rhs32_drop(orc, dg, p):
    _rhs32(orc, dg, W.drop_2d(n=7, p=p, seed=2))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_rhs32_slab_1d(orc, dg, p):
    _rhs32(orc, dg, W.slab_1d(nx=33, p=p))


def test_rhs32_physics_and_walls(orc, dg):
    wl = W.rayleigh_taylor(n=6, p=4, seed=3)
    wl.bc = ("periodic", "periodic", "noslip", "slip")
    _rhs32(orc, dg, wl)


def test_rhs32_pressure_boundary(orc, dg):
    wl = W.rayleigh_taylor_paper(nx=4, ny=12, p=4)
    _rhs32(orc, dg, wl)


def test_fp32bulk_paper_rayleigh_taylor_tracks_fp64(orc, dg):
    """The paper's Rayleigh-Taylor domain with the pressure top, 20 steps: phi and P within 1e-5
    (relative L2) of the FP64 path."""
    wl = W.rayleigh_taylor_paper(nx=8, ny=32, p=4)
    w64 = _run(dg, wl, "fp64", 20)
    w32 = _run(dg, wl, "fp32bulk", 20)
    pb = problem(orc, wl)
    assert _l2(w32[0], w64[0]) <= 1e-5
    assert _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, w64)[3]) <= 1e-5


def test_rhs32_full_size(orc, dg):
    _rhs32(orc, dg, W.drop_2d(n=64, p=3, seed=2))


def _run(dg, wl, precision, nsteps):
    import torch
    s = dg.Solver(wl, precision=precision)
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, nsteps)
    out = d.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    return out


def _l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fp32bulk_500_steps_accuracy(orc, dg):
    """Config-2 workload, 500 SSP-RK3 steps: phi and P within 1e-5 (relative L2) of FP64."""
    wl = W.drop_2d(n=64, p=3, seed=2)
    w64 = _run(dg, wl, "fp64", 500)
    w32 = _run(dg, wl, "fp32bulk", 500)
    pb = problem(orc, wl)
    p64, p32 = orc.primitives(pb, w64), orc.primitives(pb, w32)
    e_phi = _l2(w32[0], w64[0])
    e_P = _l2(p32[3], p64[3])
    e_u = _l2(p32[1], p64[1])
    assert e_phi <= 1e-5 and e_P <= 1e-5, (e_phi, e_P, e_u)
    # a pressure error dP moves the air velocity by ~ dP/(rho c), so u is looser (reported)
    assert e_u <= 1e-3, e_u


def test_fp32bulk_slab_1000_steps_accuracy(orc, dg):
    """The 1D slab workload (100 elements, p = 3), all of its 1000 steps: phi and P within 1e-5
    (relative L2) of FP64.  With the acoustic time step a field changes by a few parts in 1e5 per
    step, so an FP32 state rounded at every stage drifts by ~1e-5 over 1000 steps; the carried
    float-float step start keeps the change's low bits."""
    wl = W.slab_1d(nx=100, p=3)
    w64 = _run(dg, wl, "fp64", 1000)
    w32 = _run(dg, wl, "fp32bulk", 1000)
    pb = problem(orc, wl)
    e_phi = _l2(w32[0], w64[0])
    e_P = _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, w64)[3])
    assert e_phi <= 1e-5 and e_P <= 1e-5, (e_phi, e_P)


def test_fp32bulk_rayleigh_taylor_2000_steps_accuracy(orc, dg):
    """The Rayleigh-Taylor set-up (walls, viscous stress, gravity, surface tension) on 64 x 64,
    p = 4, for the workload's 2000 steps: phi and P within 1e-5 (relative L2) of FP64."""
    wl = W.rayleigh_taylor(n=64, p=4, seed=3)
    w64 = _run(dg, wl, "fp64", 2000)
    w32 = _run(dg, wl, "fp32bulk", 2000)
    pb = problem(orc, wl)
    e_phi = _l2(w32[0], w64[0])
    e_P = _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, w64)[3])
    assert e_phi <= 1e-5 and e_P <= 1e-5, (e_phi, e_P)


def test_fp32bulk_short_run_against_oracle(orc, dg):
    wl = W.drop_2d(n=16, p=3, seed=2)
    w32 = _run(dg, wl, "fp32bulk", 20)
    wr = orc.rk3(problem(orc, wl), wl.w, wl.dt, 20)
    pb = problem(orc, wl)
    assert _l2(w32[0], wr[0]) <= 1e-6
    assert _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, wr)[3]) <= 1e-6


@pytest.mark.parametrize("case", [1, 2])
def test_rhs32_rising_bubble(orc, dg, case):
    _rhs32(orc, dg, W.rising_bubble(nx=4, ny=8, p=4, case=case))


def test_fp32bulk_rising_bubble_tracks_fp64(orc, dg):
    """The rising bubble on 10 x 20 quads, p = 4, 200 steps: phi and P within 1e-5 (relative L2)
    of the FP64 path."""
    wl = W.rising_bubble(nx=10, ny=20, p=4)
    w32, w64 = _run(dg, wl, "fp32bulk", 200), _run(dg, wl, "fp64", 200)
    pb = problem(orc, wl)
    assert _l2(w32[0], w64[0]) <= 1e-5
    assert _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, w64)[3]) <= 1e-5


def test_fp32bulk_rayleigh_taylor_full_size_10_steps_against_oracle(orc, dg):
    """Config 3 at full size, 10 steps in one call, against the oracle's SSP-RK3 (OpenMP build,
    bit-identical to the plain one): phi and P within 1e-6 (relative L2), as the short drop run."""
    import os
    wl = W.rayleigh_taylor(n=256, p=4, seed=3)
    w32 = _run(dg, wl, "fp32bulk", 10)
    pb = problem(orc, wl)
    wr = orc.rk3(pb, wl.w, wl.dt, 10, threads=os.cpu_count() or 1)
    assert _l2(w32[0], wr[0]) <= 1e-6
    assert _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, wr)[3]) <= 1e-6


def test_fp32bulk_conversion_round_trip_keeps_pressure(orc, dg):
    """nsteps = 0 is a no-op; one step with a tiny dt changes P by ~FP32 round-off only."""
    import torch
    wl = W.drop_2d(n=8, p=3, seed=2)
    s = dg.Solver(wl, precision="fp32bulk")
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, 0)
    assert np.array_equal(d.cpu().numpy(), wl.w)
    s.dg_step(d, 1e-14, 1)
    pb = problem(orc, wl)
    P0, P1 = orc.primitives(pb, wl.w)[3], orc.primitives(pb, d.cpu().numpy())[3]
    assert np.abs(P1 / P0 - 1).max() < 1e-6
    s.close()



def _split_merge_model(d):
    """What a call of several FP32-bulk steps hands back for an FP64 value d when every increment
    is exactly zero, written from the definitions: hi = d rounded to 24 significant bits (ties away
    from zero, at the 29th bit below the double's last place), lo = d - hi rounded to nearest float,
    result hi + lo (exact in FP64); magnitudes below 2^-74 (lo would not be a normal float) give a
    signed zero."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    b = d.view(np.uint64)
    e = (b >> np.uint64(52)) & np.uint64(0x7FF)
    low29 = b & np.uint64(0x1FFFFFFF)
    up = low29 >= np.uint64(1 << 28)
    bh = (b & ~np.uint64(0x1FFFFFFF)) + np.where(up, np.uint64(1 << 29), np.uint64(0))
    hi = bh.view(np.float64)
    assert np.array_equal(hi.astype(np.float32).astype(np.float64), hi)
    lo = (d - hi).astype(np.float32).astype(np.float64)
    out = hi + lo
    return np.where(e < 949, np.copysign(0.0, d), out)


def test_fp32bulk_fp64_state_split_and_merge(dg):
    """The integer-arithmetic split of the FP64 state into float pairs and the merge back (first and
    last launch of a call of several steps), on a state whose fields span many binades (psi from
    1e-30, below the split's 2^-74 floor, to 1e2; partial densities from 1e-3 to 1e3; phi with exact
    0 and 1): with a step size below the smallest float every FP32 increment is exactly zero, so the
    call must hand back exactly the model's hi + lo for phi, psi, m_l and rho u; rho E, whose
    stiffened-gas constant is taken off and put back in FP64, to a few ulps of rho E and Cmix."""
    import torch
    wl = W.drop_2d(n=8, p=3, seed=2)
    rng = np.random.default_rng(11)
    N = wl.N
    phi = rng.uniform(0.0, 1.0, N)
    phi[::17] = 0.0
    phi[5::17] = 1.0
    psi = rng.choice([-1.0, 1.0], N) * 10.0 ** rng.uniform(-30, 2, N)
    m1 = 10.0 ** rng.uniform(-3, 3, N)
    m2 = 10.0 ** rng.uniform(-3, 3, N)
    rho = m1 + m2
    u, v = rng.uniform(-10, 10, N), rng.uniform(-10, 10, N)
    P = 10.0 ** rng.uniform(0, 6, N)
    C = [wl.gamma[l] * wl.pinf[l] / (wl.gamma[l] - 1) for l in range(2)]
    Cmix = phi * C[0] + (1 - phi) * C[1]
    G = phi / (wl.gamma[0] - 1) + (1 - phi) / (wl.gamma[1] - 1)
    rE = 0.5 * rho * (u * u + v * v) + Cmix + P * G
    w = np.stack([phi, psi, m1, m2, rho * u, rho * v, rE])
    s = dg.Solver(wl, precision="fp32bulk")
    d = torch.from_numpy(w.copy()).cuda()
    s.dg_step(d, 1e-300, 3)
    got = d.cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    for k in range(6):
        want = _split_merge_model(w[k])
        # exact equality (the sign of a zero may differ: a zero increment's sign enters the float sum)
        assert np.array_equal(got[k], want), (k, np.abs(got[k] - want).max())
    assert np.any(got[1] == 0.0) and np.any(got[1] != 0.0)
    # rho E: Cmix(phi) taken off in FP64, the rest split and merged, Cmix(phi out) put back
    dC, C2 = C[0] - C[1], C[1]
    red = rE - (dC * phi + C2)
    want = _split_merge_model(red) + (dC * got[0] + C2)
    tol = 8 * np.finfo(np.float64).eps * (np.abs(rE) + abs(C[0]) + abs(C[1])) + 2.0 ** -47 * np.abs(red)
    assert np.all(np.abs(got[6] - want) <= tol), np.max(np.abs(got[6] - want) / tol)


def test_fp32bulk_rayleigh_taylor_physics_tracks_fp64(orc, dg):
    """Walls, viscous stress, gravity and surface tension in the FP32-bulk path: 20 steps of a
    32 x 32, p = 4 Rayleigh-Taylor set-up stay within 1e-5 (relative L2) of the FP64 path in
    phi and P."""
    wl = W.rayleigh_taylor(n=32, p=4, seed=3)
    w64 = _run(dg, wl, "fp64", 20)
    w32 = _run(dg, wl, "fp32bulk", 20)
    pb = problem(orc, wl)
    assert _l2(w32[0], w64[0]) <= 1e-5
    assert _l2(orc.primitives(pb, w32)[3], orc.primitives(pb, w64)[3]) <= 1e-5


@pytest.mark.parametrize("make,nsteps", [
    (lambda: W.drop_2d(n=12, p=3, seed=2), 11),      # one 8-step graph + a 3-step graph
    (lambda: W.drop_2d(n=9, p=5, seed=7), 2),         # the 2-step remainder graph alone
    (lambda: W.rayleigh_taylor(n=8, p=4, seed=3), 9),  # walls, viscous, gravity, surface tension
    (lambda: W.slab_1d(nx=40, p=3), 5),
    # grids of several waves: the plain-launch kernel variants (the cases above fit on the GPU at
    # once and run as programmatic dependent launches)
    (lambda: W.drop_2d(n=128, p=3, seed=2), 3),
    (lambda: W.rayleigh_taylor(n=128, p=4, seed=3), 2),
])
def test_fp32bulk_multi_step_call_matches_single_steps(orc, dg, make, nsteps):
    """n steps in one call keep the FP32 step start (hi, lo) between steps and fuse the surface part
    of each stage with the volume part of the next; n calls of one step write the FP64 state and
    split it again at every step boundary.  hi + lo survives that round trip except for the FP64
    rounding of rho E + Cmix(phi), which can move hi by one FP32 unit where lo sits at half a unit;
    the right-hand side reads hi, so the two agree to FP32 rounding plus the effect of one unit of
    the stored pressure on the pressure gradient: per variable
    max |a - b| <= 1e-6 max |b| + 3 n dt 4 eps32 max|P| (2/h) max_i sum_c |D_ic| (momentum, times
    max|u| for the energy)."""
    import torch
    wl = make()
    s = dg.Solver(wl, precision="fp32bulk")
    a = torch.from_numpy(wl.w.copy()).cuda()
    b = a.clone()
    s.dg_step(a, wl.dt, nsteps)
    for _ in range(nsteps):
        s.dg_step(b, wl.dt, 1)
    assert s.dg_status_read() == 0
    s.close()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert not np.array_equal(b, wl.w)
    prim = orc.primitives(problem(orc, wl), b)
    xi, _ = orc.gll(wl.p)
    D = orc.lagrange_deriv(wl.p, xi)
    dP = 4 * np.finfo(np.float32).eps * np.abs(prim[3]).max() * (2.0 / min(wl.hx, wl.hy)) * np.abs(D).sum(axis=1).max()
    umax = np.max(np.hypot(prim[1], prim[2]))
    extra = {4: dP, 5: dP, 6: dP * umax}
    for v in range(7):
        sc = np.abs(b[v]).max()
        tol = 1e-6 * max(sc, 1e-30) + 3 * nsteps * wl.dt * extra.get(v, 0.0)
        assert np.abs(a[v] - b[v]).max() <= tol, (v, np.abs(a[v] - b[v]).max(), sc, tol)


def test_step_launch_counts(dg):
    """dg_step_launches: FP64 six launches a step, FP32-bulk 1 + 3 n (inviscid and viscous)."""
    for wl in (W.rayleigh_taylor(n=6, p=4), W.drop_2d(n=6, p=3)):
        s64, s32 = dg.Solver(wl), dg.Solver(wl, precision="fp32bulk")
        assert [s64.dg_step_launches(n) for n in (0, 1, 4)] == [0, 6, 24]
        assert [s32.dg_step_launches(n) for n in (0, 1, 4)] == [0, 4, 13]
        s64.close()
        s32.close()
