"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, entry by entry.

Tolerance (FP64 path): for every variable v,
    max_n |L_gpu - L_orc| <= 1e-12 * max_n S_v   and   ||L_gpu - L_orc||_2 <= 1e-12 ||S_v||_2,
where S (from the oracle) is the M^-1-scaled sum of the absolute values of every
contribution to R: the scale of the terms that cancel (in equilibrium regions L ~ 0).
The pressure, whose recovery cancels about four digits, is evaluated in the same
IEEE operation order on both sides, so the bound holds for the P-dependent terms too.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rhs_both(orc, dg, wl, w=None):
    import torch
    w = wl.w if w is None else w
    L_ref, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    solver = dg.Solver(wl)
    L = solver.dg_rhs(torch.from_numpy(np.array(w)).cuda()).cpu().numpy()
    assert solver.dg_status_read() == 0
    solver.close()
    return L, L_ref, S


def _assert_parity(L, L_ref, S, tol=TOL):
    for v in range(7):
        s_inf = S[v].max()
        if s_inf == 0:
            assert np.abs(L[v]).max() == 0, v
            continue
        e_inf = np.abs(L[v] - L_ref[v]).max() / s_inf
        e_2 = np.linalg.norm(L[v] - L_ref[v]) / np.linalg.norm(S[v])
        assert e_inf <= tol and e_2 <= tol, (v, e_inf, e_2)


def _broken(wl, seed=4, amp=0.05):
    """Independent per-node perturbations of the primitive fields (phi, psi, P, u, v), written
    back in conserved form: every trace jumps across every face, and the state stays physical."""
    import oracle
    rng = np.random.default_rng(seed)
    prim = oracle.primitives(oracle.Problem(**wl.problem_kwargs()), wl.w)
    phi = np.clip(wl.w[0] + amp * rng.uniform(-1, 1, wl.N), 0.0, 1.0)
    psi = wl.w[1] + amp * rng.uniform(-1, 1, wl.N)
    P = prim[3] * (1 + 0.02 * rng.uniform(-1, 1, wl.N))
    u = prim[1] * (1 + 0.05 * rng.uniform(-1, 1, wl.N)) + 0.01 * rng.uniform(-1, 1, wl.N)
    v = prim[2] * (1 + 0.05 * rng.uniform(-1, 1, wl.N)) + 0.01 * rng.uniform(-1, 1, wl.N)
    return W.conserved(wl, phi, psi, P, u, v)


# ----------------------------------------------------------------------------- rhs parity

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_rhs_1d_slab(orc, dg, p):
    wl = W.slab_1d(nx=37, p=p)  # 37 elements: ragged last block
    _assert_parity(*_rhs_both(orc, dg, wl))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_rhs_2d_drop_orders(orc, dg, p):
    wl = W.drop_2d(n=7, p=p, seed=2)  # 49 elements: several tiles and a ragged tail
    _assert_parity(*_rhs_both(orc, dg, wl))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_rhs_discontinuous_state(orc, dg, p):
    wl = W.drop_2d(n=6, p=p, seed=5)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


def test_rhs_air_bubble_in_water(orc, dg):
    wl = W.drop_2d(n=8, p=3, seed=9, water_inside=False, R=0.2)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


def test_rhs_non_square_elements(orc, dg):
    wl = W.Workload(name="rect", dim=2, nx=5, ny=3, p=3, x0=-0.5, x1=1.5, y0=0.0, y1=0.6, Gamma=1.3, eps=0.04)
    x, y = W.node_coords(wl)
    s = np.hypot(x - 0.4, y - 0.3) - 0.2
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, 0.7, -0.4)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 3), (2, 1)])
def test_rhs_self_periodic_tiny_meshes(orc, dg, nx, ny):
    wl = W.Workload(name="tiny", dim=2, nx=nx, ny=ny, p=3, Gamma=1.0, eps=0.1)
    x, y = W.node_coords(wl)
    s = np.hypot(x - 0.5, y - 0.5) - 0.25
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, 0.4, 0.3)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


@pytest.mark.parametrize("bc", ["noslip", "slip"])
def test_rhs_walls(orc, dg, bc):
    wl = W.Workload(name="box", dim=2, nx=5, ny=4, p=3, bc=(bc,) * 4, Gamma=1.0, eps=0.05)
    x, y = W.node_coords(wl)
    u = 0.3 + np.sin(np.pi * x) * np.cos(np.pi * y)
    v = -0.2 - np.cos(np.pi * x) * np.sin(np.pi * y)
    s = np.hypot(x - 0.4, y - 0.55) - 0.2
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, u, v)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


@pytest.mark.parametrize("side", [0, 3])
def test_rhs_pressure_boundary(orc, dg, side):
    """The Riemann-invariant boundary at rest at constant pressure (Sec. 4.2) on one side, walls
    elsewhere, with a moving, discontinuous state and a pressure different from the interior."""
    bc = ["slip"] * 4
    bc[side] = "pressure"
    pbc = [0.0] * 4
    pbc[side] = 0.9e5
    wl = W.Workload(name="pbox", dim=2, nx=5, ny=4, p=3, bc=tuple(bc), p_bc=tuple(pbc), Gamma=1.0, eps=0.05)
    x, y = W.node_coords(wl)
    u = 0.3 + np.sin(np.pi * x) * np.cos(np.pi * y)
    v = -0.2 - np.cos(np.pi * x) * np.sin(np.pi * y)
    s = np.hypot(x - 0.4, y - 0.55) - 0.2
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, u, v)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


def test_rhs_paper_rayleigh_taylor_domain(orc, dg):
    """The paper's Rayleigh-Taylor domain [0, 1] x [0, 4]: slip sides, no-slip bottom, pressure
    top, viscous stress and gravity."""
    wl = W.rayleigh_taylor_paper(nx=4, ny=12, p=3)
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


def test_step_paper_rayleigh_taylor_domain(orc, dg):
    wl = W.rayleigh_taylor_paper(nx=4, ny=12, p=3)
    w, w_ref = _step_both(orc, dg, wl, 5)
    _assert_steps_close(orc, wl, 5, w, w_ref)


@pytest.mark.parametrize("visc,st,grav", [(True, False, False), (False, True, False), (False, False, True),
                                          (True, True, True)])
def test_rhs_physics_terms(orc, dg, visc, st, grav):
    wl = W.rayleigh_taylor(n=6, p=4, seed=3)
    wl.viscous, wl.surface_tension, wl.gravity = visc, st, grav
    wl.bc = ("periodic", "periodic", "noslip", "slip")
    _assert_parity(*_rhs_both(orc, dg, wl, _broken(wl)))


def test_rhs_full_size_drop_64x64_p3(orc, dg):
    wl = W.drop_2d(n=64, p=3, seed=2)
    _assert_parity(*_rhs_both(orc, dg, wl))


def test_rhs_full_size_rayleigh_taylor_256x256_p4(orc, dg):
    wl = W.rayleigh_taylor(n=256, p=4, seed=3)
    _assert_parity(*_rhs_both(orc, dg, wl))


# ----------------------------------------------------------------------------- step parity

def _step_both(orc, dg, wl, nsteps, w=None):
    import torch
    w = wl.w if w is None else w
    w_ref = orc.rk3(problem(orc, wl), w, wl.dt, nsteps)
    solver = dg.Solver(wl)
    d = torch.from_numpy(np.array(w)).cuda()
    solver.dg_step(d, wl.dt, nsteps)
    out = d.cpu().numpy()
    assert solver.dg_status_read() == 0
    solver.close()
    return out, w_ref


def _kappa_P(orc, wl, w):
    """Condition number of the stiffened-gas pressure recovery,
    max (|rho E| + |Cmix| + |rho k|) / |P sum phi_l/(gamma_l-1)|: a one-ulp change of rho E
    moves P by kappa_P ulps of P."""
    prim = orc.primitives(problem(orc, wl), w)
    g1, g2 = wl.gamma
    C = [wl.gamma[l] * wl.pinf[l] / (wl.gamma[l] - 1.0) for l in range(2)]
    phi = w[0]
    Cm = np.abs(phi * C[0] + (1 - phi) * C[1])
    Gm = phi / (g1 - 1) + (1 - phi) / (g2 - 1)
    rhok = 0.5 * (w[4] ** 2 + w[5] ** 2) / (w[2] + w[3])
    return float(np.max((np.abs(w[6]) + Cm + rhok) / np.abs(prim[3] * Gm)))


def _assert_steps_close(orc, wl, nsteps, w, w_ref):
    """Multi-step bound.  Per right-hand side the two sides agree to 1e-12 of the term scale S,
    but a one-ulp difference of rho E after a stage moves P by kappa_P ulps, which drives the
    next stage; so after n stages the states may differ by ~ n kappa_P eps relative to
    max|w| + nsteps dt max S.  The bound allows 4 eps per stage."""
    L, S = orc.rhs(problem(orc, wl), wl.w, want_scale=True)
    kappa = _kappa_P(orc, wl, wl.w)
    tol = max(1e-12, 3 * nsteps * kappa * 4 * np.finfo(float).eps)
    for v in range(7):
        scale = np.abs(w_ref[v]).max() + nsteps * wl.dt * S[v].max()
        err = np.abs(w[v] - w_ref[v]).max() / scale
        assert err <= tol, (v, err, tol)


def test_one_step_parity(orc, dg):
    """A single SSP-RK3 step (three right-hand sides and stage updates) from the same state."""
    wl = W.drop_2d(n=12, p=3, seed=2)
    w, w_ref = _step_both(orc, dg, wl, 1)
    _assert_steps_close(orc, wl, 1, w, w_ref)


def test_step_1d_slab_100_steps(orc, dg):
    wl = W.slab_1d(nx=100, p=3)
    w, w_ref = _step_both(orc, dg, wl, 100)
    _assert_steps_close(orc, wl, 100, w, w_ref)


def test_step_drop_graph_unroll_remainder(orc, dg):
    """11 steps = one 8-step graph + three 1-step graphs."""
    wl = W.drop_2d(n=8, p=3, seed=2)
    w, w_ref = _step_both(orc, dg, wl, 11)
    _assert_steps_close(orc, wl, 11, w, w_ref)


def test_step_full_size_drop(orc, dg):
    wl = W.drop_2d(n=64, p=3, seed=2)
    w, w_ref = _step_both(orc, dg, wl, 3)
    _assert_steps_close(orc, wl, 3, w, w_ref)


def test_step_full_size_rayleigh_taylor_10_steps(orc, dg):
    """Config 3 at full size (256 x 256, p = 4, viscous, gravity, surface tension, no-slip walls):
    10 SSP-RK3 steps against the oracle's (its OpenMP build on every host core, bit-identical to
    the plain one), within the multi-step bound."""
    import os
    import torch
    wl = W.rayleigh_taylor(n=256, p=4, seed=3)
    w_ref = orc.rk3(problem(orc, wl), wl.w, wl.dt, 10, threads=os.cpu_count() or 1)
    solver = dg.Solver(wl)
    d = torch.from_numpy(wl.w.copy()).cuda()
    solver.dg_step(d, wl.dt, 10)
    w = d.cpu().numpy()
    assert solver.dg_status_read() == 0
    solver.close()
    _assert_steps_close(orc, wl, 10, w, w_ref)


@pytest.mark.parametrize("case", [1, 2])
def test_rhs_rising_bubble(orc, dg, case):
    """The paper's rising bubble (slip sides, no-slip bottom, pressure top, viscous, gravity,
    surface tension; both cases) on 4 x 8 quads, p = 4."""
    _assert_parity(*_rhs_both(orc, dg, W.rising_bubble(nx=4, ny=8, p=4, case=case)))


def test_step_rising_bubble(orc, dg):
    wl = W.rising_bubble(nx=4, ny=8, p=4)
    w, w_ref = _step_both(orc, dg, wl, 5)
    _assert_steps_close(orc, wl, 5, w, w_ref)


def test_step_rayleigh_taylor_small(orc, dg):
    wl = W.rayleigh_taylor(n=8, p=4, seed=3)
    w, w_ref = _step_both(orc, dg, wl, 5)
    _assert_steps_close(orc, wl, 5, w, w_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
def test_step_graphs_of_several_state_arrays(dg, precision):
    """A context keeps the step graphs of the two state arrays used most recently: stepping three
    buffers in turn (the third evicts the least recently used graphs, which are captured again
    later) gives, for each buffer, exactly what a context of its own gives."""
    import torch
    wls = [W.drop_2d(n=6, p=3, seed=k) for k in (1, 2, 3)]
    s = dg.Solver(wls[0], precision=precision)
    bufs = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    dt = wls[0].dt
    for order in ((0, 1), (0, 1), (2, 0), (1, 2), (0,)):
        for k in order:
            s.dg_step(bufs[k], dt, 3)
    counts = [4, 3, 2]  # calls of 3 steps per buffer
    s.close()
    for k in range(3):
        ref_s = dg.Solver(wls[0], precision=precision)
        ref = torch.from_numpy(wls[k].w.copy()).cuda()
        for _ in range(counts[k]):
            ref_s.dg_step(ref, dt, 3)
        ref_s.close()
        assert torch.equal(bufs[k], ref), k


def test_step_zero_is_noop(dg):
    import torch
    wl = W.drop_2d(n=4, p=2, seed=1)
    s = dg.Solver(wl)
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, 0)
    assert np.array_equal(d.cpu().numpy(), wl.w)
    s.close()


def test_stream_handle_is_torch_current_stream(dg):
    """The binding passes torch's current stream (the default one, or one made current with
    torch.cuda.stream) to the library."""
    import torch
    from paper_2306_05002_gb300 import _stream
    assert _stream().value == (torch.cuda.current_stream().cuda_stream or None)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert _stream().value == s.cuda_stream
    assert _stream(s).value == s.cuda_stream
    assert _stream().value == (torch.cuda.current_stream().cuda_stream or None)


@pytest.mark.parametrize("precision,pinned,maker", [
    ("fp64", False, "drop"), ("fp64", True, "drop"), ("fp32bulk", False, "drop"), ("fp32bulk", True, "drop"),
    ("fp32bulk", True, "rt"), ("fp32bulk", True, "drop64")])
def test_step_host_buffer_round_trip(orc, dg, precision, pinned, maker):
    """dg_step_host (a CPU tensor, pageable or pinned) gives exactly dg_step on a device copy, and
    the FP64 result matches the oracle.  Single-step calls come first: on a pinned state the
    FP32-bulk single step reads the state over the host link once, keeps a device copy and adds its
    last increment to that copy (the same FP64 arithmetic as on a device state)."""
    import torch
    wl = {"drop": lambda: W.drop_2d(n=5, p=3, seed=2), "rt": lambda: W.rayleigh_taylor(n=6, p=4),
          "drop64": lambda: W.drop_2d(n=64, p=3, seed=2)}[maker]()  # drop64: the end-to-end workload
    s = dg.Solver(wl, precision=precision)
    h = torch.from_numpy(wl.w.copy())
    if pinned:
        h = h.pin_memory()
    d = torch.from_numpy(wl.w.copy()).cuda()
    for k in (1, 1, 2, 3):  # the staging buffer and the device copy are reused
        s.dg_step(h, wl.dt, k)
        s.dg_step(d, wl.dt, k)
        assert np.array_equal(h.numpy(), d.cpu().numpy()), k
    assert s.dg_status_read() == 0
    s.close()
    if precision == "fp64":
        _assert_steps_close(orc, wl, 7, h.numpy(), orc.rk3(problem(orc, wl), wl.w, wl.dt, 7))


# ----------------------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("maker", [lambda: W.drop_2d(n=9, p=3, seed=2), lambda: W.slab_1d(nx=40, p=4),
                                   lambda: W.rayleigh_taylor(n=6, p=4)])
def test_diag_matches_oracle(orc, dg, maker):
    import torch
    wl = maker()
    ref = orc.diag(problem(orc, wl), wl.w)
    s = dg.Solver(wl)
    got = np.array(s.dg_diag(torch.from_numpy(wl.w.copy()).cuda()))
    s.close()
    np.testing.assert_allclose(got[:7], ref[:7], rtol=1e-13, atol=1e-13 * np.abs(ref[:7]).max())
    np.testing.assert_array_equal(got[7:9], ref[7:9])   # min/max phi are exact
    np.testing.assert_array_equal(got[9:11], ref[9:11])  # P is reproduced bit for bit
    np.testing.assert_allclose(got[11:15], ref[11:15], rtol=1e-15, atol=1e-300)
    assert got[15] == ref[15] == 0


def test_nonfinite_flag(dg):
    import torch
    wl = W.drop_2d(n=4, p=3, seed=1)
    w = wl.w.copy()
    w[6, 5] = np.nan
    s = dg.Solver(wl)
    s.dg_rhs(torch.from_numpy(w).cuda())
    assert s.dg_status_read() == -5
    assert s.dg_status_read() == 0  # cleared
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
def test_step_size_changes_between_calls(dg, precision):
    """The captured step graphs read dt from device memory: calls with alternating step sizes on one
    context give exactly what fresh contexts give for each sequence of step sizes."""
    import torch
    wl = W.drop_2d(n=8, p=3, seed=3)
    dts = [wl.dt, 0.5 * wl.dt, wl.dt, 0.25 * wl.dt]
    s = dg.Solver(wl, precision=precision)
    a = torch.from_numpy(wl.w.copy()).cuda()
    for k, dt in enumerate(dts):
        s.dg_step(a, dt, 1 + k % 3)  # single steps and multi-step graphs
    s.close()
    b = torch.from_numpy(wl.w.copy()).cuda()
    for k, dt in enumerate(dts):
        f = dg.Solver(wl, precision=precision)
        f.dg_step(b, dt, 1 + k % 3)
        f.close()
    assert torch.equal(a, b)


def test_peak_flops_probe(dg):
    """The FMA-chain probe behind the FP64 rooflines: positive, FP64 within the range GB300-class
    parts have (0.1 to 100 TFLOP/s) and FP32 well above FP64 (the reduced FP64 pipe)."""
    f64 = dg.peak_flops("fp64")
    f32 = dg.peak_flops("fp32")
    assert 0.1 < f64 < 100.0, f64
    assert f32 > 10.0 * f64, (f32, f64)
