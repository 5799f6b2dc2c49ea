"""Pins of the oracle's wall treatment (Sec. 4.2 boundaries, Sec. 2 viscous stress) and of its
degenerate-normal branch, against closed forms that hold only for the right ghost states:

* slip walls: a uniform flow along a slip channel is exactly steady; a slip wall lets no mass
  or energy through and exerts no tangential force, whatever the flow;
* no-slip viscous walls: plane Poiseuille flow driven by gravity is exactly steady in mass and
  momentum, and its energy gains exactly the viscous dissipation mu (du/dy)^2; the wall penalty
  of a uniform flow is eta mu (u+ - u-) with the mirrored ghost velocity;
* n = 0 where grad psi vanishes: with a constant level set the phase-field equation at rest is
  the linear interior-penalty diffusion of a_1 = Gamma eps grad phi.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import mass_weights, problem, uniform_state


def _channel(bc, p=3, n=3, **kw):
    """x periodic, walls of kind `bc` at y = 0 and y = 1."""
    return W.Workload(name="ch", dim=2, nx=n, ny=n, p=p, bc=("periodic", "periodic", bc, bc), **kw)


# --------------------------------------------------------------------------- slip walls

@pytest.mark.parametrize("viscous", [False, True])
def test_slip_channel_uniform_flow_is_steady(orc, viscous):
    """Uniform (U, 0) between slip walls at y = 0, 1: the ghost equals the own state (only the
    normal velocity, zero here, is reversed), so every face flux is the physical flux and L = 0
    to round-off -- with or without viscosity.  A no-slip channel is not steady (drag)."""
    kw = dict(Gamma=0.5, eps=0.02, viscous=viscous, mu=(1e-2, 2e-2) if viscous else (0.0, 0.0))
    wl = _channel("slip", **kw)
    w = uniform_state(wl, 0.35, 1e5, 0.8, 0.0, psi=0.2)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    for v in range(7):
        assert np.abs(L[v]).max() <= 1e-13 * S.max(), v
    wl_ns = _channel("noslip", **kw)
    L_ns = orc.rhs(problem(orc, wl_ns), w)
    assert np.abs(L_ns[4]).max() > 1e3 * 1e-13 * S.max()


def test_slip_channel_rotated_uniform_flow_is_steady(orc):
    """The same with the walls at x = 0, 1 and the flow along y."""
    wl = W.Workload(name="ch", dim=2, nx=3, ny=4, p=2, bc=("slip", "slip", "periodic", "periodic"),
                    Gamma=0.5, eps=0.02)
    w = uniform_state(wl, 0.7, 1e5, 0.0, -1.1, psi=-0.4)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    assert np.abs(L).max() <= 1e-13 * S.max()


def _flow_through_walls(wl):
    """A drop in a flow whose velocity has a normal component on every wall."""
    x, y = W.node_coords(wl)
    u = 0.4 + 0.3 * np.sin(np.pi * x) * np.cos(np.pi * y)
    v = 0.25 - 0.2 * np.cos(np.pi * x) * np.sin(2 * np.pi * y)
    P = 1e5 * (1.0 + 0.01 * np.cos(np.pi * x) * np.cos(np.pi * y))
    s = np.hypot(x - 0.45, y - 0.55) - 0.2
    return W.conserved(wl, W.tanh_profile(s, wl.eps), s, P, u, v)


def test_slip_walls_pass_no_mass_or_energy(orc):
    """Box with slip walls on all sides and a flow crossing them: the reversed normal velocity
    makes the wall flux of m_1, m_2 and rho E vanish, so their integrals are conserved."""
    wl = W.Workload(name="box", dim=2, nx=4, ny=4, p=3, bc=("slip",) * 4, Gamma=1.0, eps=0.05)
    w = _flow_through_walls(wl)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    M = mass_weights(orc, wl)
    for var in (2, 3, 6):
        assert abs(np.sum(M * L[var])) < 1e-13 * np.sum(M * S[var]), var


def test_slip_walls_exert_no_tangential_force(orc):
    """Channel with slip walls at y = 0, 1 and a flow crossing them: the tangential momentum
    of the ghost equals the own, so the walls exert no x-force and int rho u is conserved;
    no-slip walls, which reverse it, do exert one."""
    wl = _channel("slip", p=3, n=4, Gamma=1.0, eps=0.05)
    w = _flow_through_walls(wl)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    M = mass_weights(orc, wl)
    assert abs(np.sum(M * L[4])) < 1e-13 * np.sum(M * S[4])
    L_ns = orc.rhs(problem(orc, _channel("noslip", p=3, n=4, Gamma=1.0, eps=0.05)), w)
    assert abs(np.sum(M * L_ns[4])) > 1e3 * 1e-13 * np.sum(M * S[4])


@pytest.mark.parametrize("bc", ["slip", "noslip"])
def test_walls_reflect_normal_momentum(orc, bc):
    """Uniform flow (0, V) into walls at y = 0, 1 (x periodic): both wall kinds reverse the normal
    momentum in the ghost, so the Lax-Friedrichs flux of rho v through the walls is
    rho V^2 + P + lambda rho u_n with u_n the own normal velocity, lambda = |V| + c: the walls push
    back with int L(rho v) = -2 lambda rho V per unit length, and nothing else changes."""
    V, rho = 0.2, 1.2
    wl = _channel(bc, p=3, n=3, gamma=(1.4, 1.4), pinf=(0.0, 0.0), rho0=(rho, rho), Gamma=0.0, eps=0.0)
    w = uniform_state(wl, 0.5, 1e5, 0.0, V)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    M = mass_weights(orc, wl)
    lam = V + np.sqrt(1.4 * 1e5 / rho)
    assert abs(np.sum(M * L[5]) - (-2.0 * lam * rho * V)) < 1e-12 * np.sum(M * S[5])
    assert abs(np.sum(M * L[4])) < 1e-13 * np.sum(M * S[4])


# --------------------------------------------------------------------------- no-slip viscous walls

def _poiseuille(p, mu=0.05, g=0.4, n=3):
    """Single fluid (identical phases), phi = 1/2, constant level set, gravity g along x,
    u = rho g y (1 - y) / (2 mu), v = 0, P uniform, no-slip walls at y = 0, 1."""
    wl = _channel("noslip", p=p, n=n, gamma=(1.4, 1.4), pinf=(0.0, 0.0), rho0=(1.0, 1.0), mu=(mu, mu),
                  viscous=True, gravity=True, g=(g, 0.0), Gamma=0.3, eps=0.02)
    x, y = W.node_coords(wl)
    u = g * y * (1.0 - y) / (2.0 * mu)
    w = W.conserved(wl, np.full(wl.N, 0.5), np.full(wl.N, 0.1), 1e5, u, 0.0)
    return wl, w, y


@pytest.mark.parametrize("p", [2, 3, 4])
def test_poiseuille_flow_is_steady(orc, p):
    """The quadratic profile lies in the space (p >= 2) and vanishes at the walls, so the wall
    ghost (velocity reversed, stress equal to the own) makes every face flux the physical flux;
    mu u'' + rho g = 0 then leaves mass and momentum exactly steady."""
    wl, w, _ = _poiseuille(p)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    for v in (2, 3, 4, 5):
        assert np.abs(L[v]).max() <= 1e-12 * S[v].max(), v
    # phi and psi are uniform: only the rounding of D applied to a constant remains
    assert np.abs(L[:2]).max() <= 1e-13


@pytest.mark.parametrize("p", [3, 4])
def test_poiseuille_energy_gains_viscous_dissipation(orc, p):
    """L(rho E) = d(tau_xy u)/dy + rho g u = mu (du/dy)^2 at every node: tau_xy u is a cubic,
    represented exactly for p >= 3, and nothing crosses the walls (u = 0 there)."""
    mu, g = 0.05, 0.4
    wl, w, y = _poiseuille(p, mu=mu, g=g)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    dudy = g * (1.0 - 2.0 * y) / (2.0 * mu)
    ref = mu * dudy ** 2
    assert np.abs(L[6] - ref).max() <= 1e-11 * S[6].max()
    assert np.abs(ref).max() > 1e3 * 1e-11 * S[6].max()  # the check is not vacuous


@pytest.mark.parametrize("p", [2, 3])
def test_noslip_viscous_wall_penalty(orc, p):
    """Uniform (U, 0) in a no-slip channel: the viscous flux adds eta mu (u+ - u-) = -2 eta mu U
    per unit wall length at every wall node (the mirrored ghost; tau = 0), i.e.
    M^-1 w_f (-2 eta mu U) = -2 eta mu U p (p + 1) / h_y, eta = c_ip (p+1)^2 / h_y; elsewhere and
    in the other equations viscosity changes nothing (k+ = k-)."""
    U, mu = 0.3, 0.02
    base = dict(gamma=(1.4, 1.4), pinf=(0.0, 0.0), rho0=(1.2, 1.2), Gamma=0.0, eps=0.0)
    wl0 = _channel("noslip", p=p, n=3, **base)
    wl1 = _channel("noslip", p=p, n=3, viscous=True, mu=(mu, mu), **base)
    w = uniform_state(wl0, 0.5, 1e5, U, 0.0)
    L0, S0 = orc.rhs(problem(orc, wl0), w, want_scale=True)
    L1 = orc.rhs(problem(orc, wl1), w)
    x, y = W.node_coords(wl0)
    at_wall = (np.abs(y) < 1e-12) | (np.abs(y - 1.0) < 1e-12)
    eta = wl1.c_ip * (p + 1) ** 2 / wl1.hy
    expected = np.where(at_wall, -2.0 * eta * mu * U * p * (p + 1) / wl1.hy, 0.0)
    np.testing.assert_allclose(L1[4] - L0[4], expected, rtol=1e-12, atol=1e-12 * S0[4].max())
    for v in (0, 1, 2, 3, 5, 6):
        assert np.abs(L1[v] - L0[v]).max() <= 1e-13 * S0[v].max(), v


def test_transverse_shear_wave_rhs(orc):
    """v = A sin(2 pi x), u = 0, single fluid, P uniform: L(rho v) -> mu v'' = -4 pi^2 mu v (the
    dv/dx part of the shear stress)."""
    mu, A = 0.05, 1e-3
    wl = W.Workload(name="shear", dim=2, nx=16, ny=2, p=4, gamma=(1.4, 1.4), pinf=(0.0, 0.0),
                    rho0=(1.0, 1.0), mu=(mu, mu), viscous=True, Gamma=0.0, eps=0.0)
    x, y = W.node_coords(wl)
    v = A * np.sin(2 * np.pi * x)
    w = W.conserved(wl, np.full(wl.N, 0.5), np.zeros(wl.N), 1e5, 0.0, v)
    L = orc.rhs(problem(orc, wl), w)
    ref = -4 * np.pi ** 2 * mu * v
    assert np.abs(L[5] - ref).max() < 2e-3 * np.abs(ref).max()


def test_viscous_fluxes_conserve_with_discontinuous_state(orc):
    """With viscous stress on and a state that jumps at every face, the single-valued viscous
    face fluxes ({tau}.m + eta {mu} [u], {tau.u}.m + eta {mu} [k]) still conserve rho u and rho E
    on a periodic mesh."""
    wl = W.Workload(name="vc", dim=2, nx=4, ny=4, p=3, viscous=True, mu=(0.02, 0.05), Gamma=0.8, eps=0.03)
    x, y = W.node_coords(wl)
    rng = np.random.default_rng(17)
    u = 0.5 * np.sin(2 * np.pi * y) + 0.05 * rng.uniform(-1, 1, wl.N)
    v = 0.3 * np.cos(2 * np.pi * x) + 0.05 * rng.uniform(-1, 1, wl.N)
    s = np.hypot(x - 0.5, y - 0.5) - 0.25
    phi = np.clip(W.tanh_profile(s, wl.eps) + 0.05 * rng.uniform(-1, 1, wl.N), 0.0, 1.0)
    w = W.conserved(wl, phi, s, 1e5 * (1 + 0.01 * rng.uniform(-1, 1, wl.N)), u, v)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    M = mass_weights(orc, wl)
    for var in (2, 3, 4, 5, 6):
        assert abs(np.sum(M * L[var])) < 1e-13 * np.sum(M * S[var]), var


# --------------------------------------------------------------------------- degenerate normal

def test_constant_level_set_gives_linear_diffusion(orc):
    """With psi constant its broken gradient vanishes (to rounding), n = 0, and at rest with
    uniform pressure the phase-field equation is L(phi) = div_h(Gamma eps grad phi): linear in
    phi.  With a non-degenerate level set the sharpening term phi (1 - phi) n breaks linearity."""
    wl = W.Workload(name="lin", dim=2, nx=4, ny=4, p=3, gamma=(1.4, 1.4), pinf=(0.0, 0.0),
                    rho0=(1.0, 1.0), Gamma=0.7, eps=0.03)
    x, y = W.node_coords(wl)
    fa = 0.3 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    fb = 0.2 + 0.15 * np.cos(2 * np.pi * (x + y))
    pb = problem(orc, wl)

    def Lphi(phi, psi):
        return orc.rhs(pb, W.conserved(wl, phi, psi, 1e5, 0.0, 0.0))[0]

    psi_c = np.full(wl.N, 0.37)
    La, Lb, Lab = Lphi(fa, psi_c), Lphi(fb, psi_c), Lphi(fa + fb, psi_c)
    scale = np.abs(La).max() + np.abs(Lb).max()
    assert np.abs(Lab - La - Lb).max() < 1e-11 * scale
    psi_s = x + 0.5 * y  # non-degenerate level set: the sharpening term is back
    La, Lb, Lab = Lphi(fa, psi_s), Lphi(fb, psi_s), Lphi(fa + fb, psi_s)
    assert np.abs(Lab - La - Lb).max() > 1e-3 * scale
