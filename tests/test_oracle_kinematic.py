"""Pins of the oracle's kinematic mode (Sec. 4.1: phase field and level set advected by a
prescribed velocity, classical fourth-order Runge-Kutta in time), against what the
mathematics fixes rather than against the oracle's own formulas:

* the Rider-Kothe field is divergence-free, periodic, reverses at t = T/2, vanishes at its
  centre and turns clockwise with unit speed a quarter period from it (finite differences of the
  oracle's own field, for several vortex centres);
* a pure phase stays put, a constant level set stays put (to the rounding of D's row sums);
* for a uniform velocity the discrete phase-field mass is conserved to round-off (the
  non-conservative transport integrates to the single-valued upwind flux, and every
  a_1 term sums to zero over a periodic domain), and so for the vortex, whose nodal velocity
  is the discrete curl of its stream function: that velocity reproduces the printed field
  (finite differences of the stream function), is discretely divergence-free with continuous
  normal components across faces, and converges to the analytical field at order p;
* with Gamma = 0 the phase field is transported exactly like the level set;
* with u = 0 and a constant level set the operator is the SIP diffusion alone:
  M L is symmetric, negative semi-definite, with the constants as its null space;
* translating a planar tanh slab (on which a_1 vanishes) converges at the optimal rate
  p + 1 (the paper's droplet test, Sec. 4.1);
* the time integrator is fourth order with a time-dependent velocity (which also pins the
  stage times t, t + dt/2, t + dt/2, t + dt).
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W


def _pb(orc, n, p, ny=None, L=1.0, Gamma=1.0, eps=0.05):
    return orc.Problem(dim=2, nx=n, ny=ny or n, p=p, x0=-0.5 * L, x1=0.5 * L, y0=-0.5 * L, y1=0.5 * L,
                       Gamma=Gamma, eps=eps)


def _weights(orc, pb):
    xi, wt = orc.gll(pb.p)
    hx, hy = (pb.x1 - pb.x0) / pb.nx, (pb.y1 - pb.y0) / pb.ny
    w2 = np.outer(wt, wt).ravel() * 0.25 * hx * hy
    return np.tile(w2, pb.nx * pb.ny)


def _smooth(orc, pb, seed=0):
    x, y = orc.nodes(pb)
    r = np.random.default_rng(seed).uniform(0, 2 * np.pi, 4)
    phi = 0.5 + 0.3 * np.sin(2 * np.pi * x + r[0]) * np.cos(2 * np.pi * y + r[1])
    psi = np.sin(2 * np.pi * x + r[2]) + 0.5 * np.cos(2 * np.pi * y + r[3])
    return np.stack([phi, psi])


@pytest.mark.parametrize("centre", [(0.5, 0.5), (0.0, 0.0), (0.2, -0.1)])
def test_rider_kothe_field_properties(orc, centre):
    vel = orc.Velocity("rider_kothe", T=4.0, xc=centre[0], yc=centre[1])
    rng = np.random.default_rng(3)
    h = 1e-5
    for x, y, t in rng.uniform([-0.5, -0.5, 0.0], [0.5, 0.5, 4.0], (20, 3)):
        ux = (orc.velocity_at(vel, x + h, y, t)[0] - orc.velocity_at(vel, x - h, y, t)[0]) / (2 * h)
        vy = (orc.velocity_at(vel, x, y + h, t)[1] - orc.velocity_at(vel, x, y - h, t)[1]) / (2 * h)
        assert abs(ux + vy) < 1e-8
        u, v = orc.velocity_at(vel, x, y, t)
        assert np.allclose(orc.velocity_at(vel, x + 1.0, y - 1.0, t), (u, v), atol=1e-12)
        ur, vr = orc.velocity_at(vel, x, y, 4.0 - t)
        assert abs(u + ur) < 1e-12 and abs(v + vr) < 1e-12       # reversal about T/2
    # clockwise: unit speed +x a quarter period below the centre and -x above it; the field
    # vanishes at the centre and at t = T/2
    xc, yc = centre
    assert np.allclose(orc.velocity_at(vel, xc, yc - 0.25, 0.0), (1.0, 0.0), atol=1e-15)
    assert np.allclose(orc.velocity_at(vel, xc, yc + 0.25, 0.0), (-1.0, 0.0), atol=1e-15)
    assert np.allclose(orc.velocity_at(vel, xc, yc, 0.7), (0.0, 0.0), atol=1e-15)
    assert np.allclose(orc.velocity_at(vel, 0.3, 0.1, 2.0), (0.0, 0.0), atol=1e-15)
    assert orc.velocity_at(orc.Velocity("uniform", u0=0.3, v0=-0.7), 0.1, 0.2, 9.0) == (0.3, -0.7)


@pytest.mark.parametrize("kind", ["uniform", "rider_kothe"])
def test_pure_phase_and_constant_level_set_are_steady(orc, kind):
    pb = _pb(orc, 4, 3)
    vel = orc.Velocity(kind, u0=0.7, v0=-0.4)
    w = _smooth(orc, pb)
    w[0] = 0.0
    assert np.all(orc.kin_rhs(pb, vel, 0.3, w)[0] == 0.0)
    # a constant 1 is annihilated by D up to the rounding of its row sums
    w[0] = 1.0
    assert np.abs(orc.kin_rhs(pb, vel, 0.3, w)[0]).max() < 1e-12
    w = _smooth(orc, pb)
    w[1] = 0.37
    assert np.abs(orc.kin_rhs(pb, vel, 0.3, w)[1]).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 4])
def test_uniform_velocity_conserves_phase_field_mass(orc, p):
    pb = _pb(orc, 5, p, ny=4)
    vel = orc.Velocity("uniform", u0=0.8, v0=-0.45)
    w = _smooth(orc, pb, seed=p)
    L, S = orc.kin_rhs(pb, vel, 0.0, w, want_scale=True)
    M = _weights(orc, pb)
    assert abs(np.sum(M * L[0])) <= 1e-13 * np.sum(M * S[0])
    assert abs(np.sum(M * L[1])) <= 1e-13 * np.sum(M * S[1])


@pytest.mark.parametrize("centre", [(0.5, 0.5), (0.0, 0.0), (0.2, -0.1)])
def test_stream_function_gives_the_vortex(orc, centre):
    """u = dPsi/dy and v = -dPsi/dx (central differences of the stream function) reproduce the
    Rider-Kothe field of orc_velocity_at."""
    vel = orc.Velocity("rider_kothe", T=4.0, xc=centre[0], yc=centre[1])
    h = 1e-5
    for x, y, t in np.random.default_rng(8).uniform([-0.5, -0.5, 0.0], [0.5, 0.5, 4.0], (20, 3)):
        u = (orc.stream_at(vel, x, y + h, t) - orc.stream_at(vel, x, y - h, t)) / (2 * h)
        v = -(orc.stream_at(vel, x + h, y, t) - orc.stream_at(vel, x - h, y, t)) / (2 * h)
        assert np.allclose((u, v), orc.velocity_at(vel, x, y, t), rtol=0, atol=1e-9)


def _element_derivatives(orc, pb, f):
    """d f/dx and d f/dy of nodal values f with each element's derivative matrices (node
    a = i + (p+1) j), by numpy's matrix products rather than the oracle's basis gradients."""
    xi, _ = orc.gll(pb.p)
    D = orc.lagrange_deriv(pb.p, xi)
    P1 = pb.p + 1
    hx, hy = (pb.x1 - pb.x0) / pb.nx, (pb.y1 - pb.y0) / pb.ny
    F = f.reshape(-1, P1, P1)                       # [element][j][i]
    fx = np.einsum("ic,ejc->eji", D, F) * (2 / hx)
    fy = np.einsum("jc,eci->eji", D, F) * (2 / hy)
    return fx.reshape(-1), fy.reshape(-1)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_nodal_vortex_velocity(orc, p):
    """The scheme's nodal Rider-Kothe velocity: discretely divergence-free in every element, its
    normal component continuous across every face, and converging to the analytical field at
    order p (the derivative of a degree-p interpolant)."""
    vel = orc.Velocity("rider_kothe", T=4.0)
    errs = []
    for n in (6, 12):
        pb = _pb(orc, n, p)
        u, v = orc.kin_velocity(pb, vel, 0.7)
        ux, _ = _element_derivatives(orc, pb, u)
        _, vy = _element_derivatives(orc, pb, v)
        assert np.abs(ux + vy).max() <= 1e-12 * np.abs(ux).max()
        P1 = p + 1
        U, V = u.reshape(n, n, P1, P1), v.reshape(n, n, P1, P1)    # [ey][ex][j][i]
        assert np.abs(U[:, :, :, -1] - np.roll(U, -1, axis=1)[:, :, :, 0]).max() <= 1e-13   # E | W
        assert np.abs(V[:, :, -1, :] - np.roll(V, -1, axis=0)[:, :, 0, :]).max() <= 1e-13   # N | S
        x, y = orc.nodes(pb)
        exact = np.array([orc.velocity_at(vel, a, b, 0.7) for a, b in zip(x, y)]).T
        errs.append(max(np.abs(u - exact[0]).max(), np.abs(v - exact[1]).max()))
    assert np.log2(errs[0] / errs[1]) > p - 0.5, errs


@pytest.mark.parametrize("p", [2, 3, 4])
def test_vortex_conserves_phase_field_mass(orc, p):
    """With the discretely divergence-free vortex the phase field's mass is conserved to
    round-off, as for a uniform velocity."""
    pb = _pb(orc, 5, p, ny=4)
    vel = orc.Velocity("rider_kothe", T=4.0, xc=0.1, yc=-0.2)
    w = _smooth(orc, pb, seed=p)
    M = _weights(orc, pb)
    for t in (0.3, 1.7):
        L, S = orc.kin_rhs(pb, vel, t, w, want_scale=True)
        assert abs(np.sum(M * L[0])) <= 1e-13 * np.sum(M * S[0])


def test_phase_field_without_a1_is_transported_like_the_level_set(orc):
    pb = _pb(orc, 4, 3, Gamma=0.0)
    for vel in (orc.Velocity("uniform", u0=0.6, v0=0.9), orc.Velocity("rider_kothe", T=4.0)):
        w = _smooth(orc, pb, seed=5)
        w[1] = w[0]
        L = orc.kin_rhs(pb, vel, 0.7, w)
        assert np.array_equal(L[0], L[1])


@pytest.mark.parametrize("p,n", [(1, 4), (2, 3), (3, 2)])
def test_sip_diffusion_operator_symmetric_negative_semidefinite(orc, p, n):
    """u = 0 and a constant level set (n = 0): the phase-field operator is Gamma eps times the
    SIP Laplacian.  Columns of M L by unit vectors form a symmetric, negative semi-definite
    matrix whose null space holds the constants."""
    pb = _pb(orc, n, p, eps=0.1, Gamma=0.7)
    vel = orc.Velocity("uniform", u0=0.0, v0=0.0)
    N = pb.N
    M = _weights(orc, pb)
    A = np.zeros((N, N))
    for j in range(N):
        w = np.zeros((2, N))
        w[0, j] = 1.0
        A[:, j] = M * orc.kin_rhs(pb, vel, 0.0, w)[0]
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-12 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-11 * scale
    assert np.abs(A @ np.ones(N)).max() <= 1e-12 * scale
    assert np.sum(ev > -1e-10 * scale) == 1


def _slab(x, t, eps):
    """Planar slab of phase 1, |x - t| < 0.25 on the periodic unit interval, with the signed
    distance psi growing into it; a_1 vanishes on this profile away from the kinks of psi."""
    s = 0.25 - np.abs(((x - t + 0.5) % 1.0) - 0.5)
    return W.tanh_profile(s, eps), s


@pytest.mark.parametrize("p,meshes", [(2, (16, 32)), (3, (32, 64))])
def test_translation_converges_at_p_plus_one(orc, p, meshes):
    """eps = 0.02 keeps phi(1 - phi) below 4e-6 at the kinks of psi; p = 3 needs h < eps to be
    in the asymptotic range."""
    eps, T = 0.02, 0.05
    errs = []
    for n in meshes:
        pb = orc.Problem(dim=2, nx=n, ny=1, p=p, x0=-0.5, x1=0.5, y0=-0.5, y1=0.5, Gamma=1.0, eps=eps)
        x, _ = orc.nodes(pb)
        phi, psi = _slab(x, 0.0, eps)
        h, q = 1.0 / n, 2 * p + 1
        dt = min(0.3 * h / q, 0.1 * h * h / (q * q * eps))
        nst = int(np.ceil(T / dt))
        w = orc.kin_rk4(pb, orc.Velocity("uniform", u0=1.0, v0=0.0), np.stack([phi, psi]), 0.0, T / nst, nst)
        phie, _ = _slab(x, T, eps)
        errs.append(np.sum(_weights(orc, pb) * np.abs(w[0] - phie)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 0.7, (errs, rate)


def test_rk4_is_fourth_order_with_a_time_dependent_velocity(orc):
    pb = _pb(orc, 4, 2, eps=0.05, Gamma=0.5)
    vel = orc.Velocity("rider_kothe", T=0.5)
    w0 = _smooth(orc, pb, seed=2)
    T = 0.04
    sols = [orc.kin_rk4(pb, vel, w0, 0.1, T / n, n) for n in (8, 16, 32)]
    d1 = np.abs(sols[0] - sols[1]).max()
    d2 = np.abs(sols[1] - sols[2]).max()
    assert 12.0 < d1 / d2 < 20.0, (d1, d2, d1 / d2)
