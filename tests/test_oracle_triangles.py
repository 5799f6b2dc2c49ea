"""Pins of the oracle's kinematic mode on triangles (the paper's mesh (b), Sec. 4.1):
phi and psi under a prescribed velocity, d(phi)/dt + u.grad(phi) = div(Gamma (eps grad phi -
phi (1 - phi) n)), d(psi)/dt + u.grad(psi) = 0, on the split-rectangle triangulation,
checked against what the mathematics fixes:

* the element mass matrix integrates products of polynomials of degree <= p exactly (closed
  forms by an independent collapsed Gauss rule of many points);
* the integral of a nodal field equals the exact integral of its polynomial over the rectangle;
* with Gamma = 0 and a uniform velocity the scheme is exact for a global polynomial of degree
  <= p on elements away from the periodic seam: L = -u.grad(f);
* a uniform velocity conserves int phi and int psi for any fields and any Gamma (flux
  single-valued, transport telescoping);
* the SIP diffusion (psi constant, so n = 0) gives M L symmetric negative semi-definite with
  constants in its null space; the upwind transport gives M L with a negative semi-definite
  symmetric part;
* with Gamma = 0 the phi and psi rows are the same operator;
* a planar tanh profile with psi its signed distance is an equilibrium of the Allen-Cahn flux:
  the residual converges to zero at a rate near p - 1, and with the normal reversed it does not;
* the time integrator is fourth order against the matrix exponential of the linear operator,
  and with a time-dependent velocity (which pins the stage times);
* a smooth periodic field translated by a uniform velocity converges under refinement
  (neighbours across the periodic seam included).
"""
import numpy as np
import pytest
import scipy.linalg as sl
from numpy.polynomial.legendre import leggauss


def _np(p):
    return (p + 1) * (p + 2) // 2


def _interior(pb, margin=1):
    """Node indices of the triangles whose cells lie at least `margin` cells from the seam."""
    Np, idx = _np(pb.p), []
    for j in range(margin, pb.ny - margin):
        for i in range(margin, pb.nx - margin):
            for t in (0, 1):
                e = 2 * (i + pb.nx * j) + t
                idx.extend(range(e * Np, (e + 1) * Np))
    return np.array(idx)


def _tri_exact(V, f, n=12):
    """int_T f over the triangle with vertices V by a collapsed (Duffy) tensor Gauss rule of n^2
    points, exact for polynomials of degree <= 2n - 2."""
    a, wa = leggauss(n)
    A, B = np.meshgrid(a, a, indexing="ij")
    r, s, w = 0.5 * (1 + A) * (1 - B) - 1, B, np.outer(wa, wa) * 0.5 * (1 - B)
    (x1, y1), (x2, y2), (x3, y3) = V
    x = x1 + 0.5 * (1 + r) * (x2 - x1) + 0.5 * (1 + s) * (x3 - x1)
    y = y1 + 0.5 * (1 + r) * (y2 - y1) + 0.5 * (1 + s) * (y3 - y1)
    det = 0.25 * abs((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1))
    return (w * f(x, y)).sum() * det


def _op_matrix(orc, pb, vel, row, psi_fill=0.0):
    """Matrix of the (linear) phi right-hand side, column j = L(e_j) with psi = psi_fill."""
    N = orc.tri_num_nodes(pb)
    A = np.zeros((N, N))
    for j in range(N):
        w = np.zeros((2, N))
        w[row, j] = 1.0
        if row == 0:
            w[1, :] = psi_fill
        A[:, j] = orc.tri_rhs(pb, vel, 0.0, w)[row]
    return A


def _block_mass(orc, pb):
    return sl.block_diag(*[orc.tri_mass(pb, e) for e in range(2 * pb.nx * pb.ny)])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_matrix_exact_for_degree_p_products(orc, p):
    pb = orc.Problem(dim=2, nx=3, ny=2, p=p, x0=-0.3, x1=0.9, y0=0.1, y1=0.7, Gamma=1.0, eps=0.05)
    x, y = orc.tri_nodes(pb)
    Np = _np(p)
    for e in (0, 1, 5):
        xe, ye = x[e * Np:(e + 1) * Np], y[e * Np:(e + 1) * Np]
        V = [(xe[0], ye[0]), (xe[p], ye[p]), (xe[-1], ye[-1])]   # corner nodes, counter-clockwise
        M = orc.tri_mass(pb, e)
        for a in range(p + 1):
            for b in range(p + 1 - a):
                for c in range(p + 1):
                    for d in range(p + 1 - c):
                        ex = _tri_exact(V, lambda X, Y: X ** (a + c) * Y ** (b + d))
                        got = (xe ** a * ye ** b) @ M @ (xe ** c * ye ** d)
                        assert abs(got - ex) < 1e-14 + 1e-13 * abs(ex), (e, a, b, c, d)


@pytest.mark.parametrize("p", [1, 3, 4])
def test_integral_of_polynomial_over_rectangle(orc, p):
    x0, x1, y0, y1 = -0.3, 0.9, 0.1, 0.7
    pb = orc.Problem(dim=2, nx=3, ny=4, p=p, x0=x0, x1=x1, y0=y0, y1=y1, Gamma=1.0, eps=0.05)
    x, y = orc.tri_nodes(pb)
    for a in range(p + 1):
        for b in range(p + 1 - a):
            ex = (x1 ** (a + 1) - x0 ** (a + 1)) / (a + 1) * (y1 ** (b + 1) - y0 ** (b + 1)) / (b + 1)
            assert abs(orc.tri_integral(pb, x ** a * y ** b) - ex) < 1e-14 + 1e-13 * abs(ex)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_uniform_transport_exact_for_global_polynomial(orc, p):
    pb = orc.Problem(dim=2, nx=4, ny=5, p=p, x0=0.0, x1=1.0, y0=0.0, y1=1.2, Gamma=0.0, eps=0.05)
    x, y = orc.tri_nodes(pb)
    u0, v0 = 0.7, -0.4
    phi = 0.3 * x ** p - 0.2 * x * y ** (p - 1) + y + 0.1
    gx = 0.3 * p * x ** (p - 1) - 0.2 * y ** (p - 1)
    gy = (-0.2 * (p - 1) * x * y ** (p - 2) if p > 1 else 0.0 * x) + 1.0
    psi = 0.5 * x - y
    L = orc.tri_rhs(pb, orc.Velocity("uniform", u0, v0), 0.0, np.stack([phi, psi]))
    I = _interior(pb)
    tol = 1e-11 * max(1.0, p ** 2)
    assert np.abs(L[0][I] + u0 * gx[I] + v0 * gy[I]).max() < tol
    assert np.abs(L[1][I] + (0.5 * u0 - v0)).max() < tol


@pytest.mark.parametrize("p", [1, 3, 4])
def test_uniform_velocity_conserves_both_fields(orc, p):
    pb = orc.Problem(dim=2, nx=3, ny=4, p=p, Gamma=0.7, eps=0.05, c_ip=2.0)
    N = orc.tri_num_nodes(pb)
    w = np.random.default_rng(p).uniform(0.0, 1.0, (2, N))
    L = orc.tri_rhs(pb, orc.Velocity("uniform", 0.7, -0.4), 0.0, w)
    scale = np.abs(L).max()
    assert abs(orc.tri_integral(pb, L[0])) < 1e-14 * scale
    assert abs(orc.tri_integral(pb, L[1])) < 1e-14 * scale


@pytest.mark.parametrize("p", [1, 2, 3])
def test_sip_diffusion_symmetric_negative_semidefinite(orc, p):
    pb = orc.Problem(dim=2, nx=3, ny=3, p=p, Gamma=0.7, eps=0.05, c_ip=2.0)
    A = _block_mass(orc, pb) @ _op_matrix(orc, pb, orc.Velocity("uniform", 0.0, 0.0), 0, psi_fill=0.3)
    s = np.abs(A).max()
    assert np.abs(A - A.T).max() < 1e-13 * s
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < 1e-13 * s and ev.min() < -0.1 * s
    assert np.abs(A @ np.ones(len(A))).max() < 1e-13 * s


@pytest.mark.parametrize("p", [1, 2, 3])
def test_upwind_transport_is_dissipative(orc, p):
    pb = orc.Problem(dim=2, nx=3, ny=3, p=p, Gamma=0.0, eps=0.05)
    vel = orc.Velocity("uniform", 0.7, -0.4)
    Mb = _block_mass(orc, pb)
    for row in (0, 1):
        A = Mb @ _op_matrix(orc, pb, vel, row)
        s = np.abs(A).max()
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        assert ev.max() < 1e-13 * s and ev.min() < -0.1 * s
        assert np.abs(A @ np.ones(len(A))).max() < 1e-13 * s


def test_phi_and_psi_rows_agree_without_phase_field_flux(orc):
    pb = orc.Problem(dim=2, nx=4, ny=3, p=3, Gamma=0.0, eps=0.05)
    N = orc.tri_num_nodes(pb)
    f = np.random.default_rng(7).standard_normal(N)
    for vel in (orc.Velocity("uniform", 0.3, 0.8), orc.Velocity("rider_kothe", T=4.0)):
        L = orc.tri_rhs(pb, vel, 0.37, np.stack([f, f]))
        assert np.abs(L[0] - L[1]).max() < 1e-13 * np.abs(L).max()


def test_planar_profile_is_allen_cahn_equilibrium(orc):
    eps, p = 0.1, 4
    nv = np.array([1.0, 2.0]) / np.sqrt(5.0)
    res, flipped = [], []
    for n in (8, 16, 32):
        pb = orc.Problem(dim=2, nx=n, ny=n, p=p, Gamma=1.0, eps=eps, c_ip=2.0)
        x, y = orc.tri_nodes(pb)
        s = nv[0] * (x - 0.5) + nv[1] * (y - 0.5)
        phi = 0.5 * (1.0 + np.tanh(s / (2.0 * eps)))
        still = orc.Velocity("uniform", 0.0, 0.0)
        I = _interior(pb, n // 8)
        res.append(np.abs(orc.tri_rhs(pb, still, 0.0, np.stack([phi, s]))[0][I]).max())
        flipped.append(np.abs(orc.tri_rhs(pb, still, 0.0, np.stack([phi, -s]))[0][I]).max())
    rates = np.log2(np.array(res[:-1]) / np.array(res[1:]))
    assert np.all(rates > 2.5), (res, rates)
    assert res[-1] < 0.01 and min(flipped) > 1.0, (res, flipped)


def test_rk4_fourth_order_against_matrix_exponential(orc):
    pb = orc.Problem(dim=2, nx=3, ny=3, p=2, Gamma=0.0, eps=0.05)
    vel = orc.Velocity("uniform", 0.7, -0.4)
    A = _op_matrix(orc, pb, vel, 0)
    x, y = orc.tri_nodes(pb)
    phi0 = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    T = 0.2
    exact = sl.expm(A * T) @ phi0
    errs = []
    for ns in (8, 16, 32):
        w = orc.tri_rk4(pb, vel, np.stack([phi0, np.zeros_like(phi0)]), 0.0, T / ns, ns)
        errs.append(np.abs(w[0] - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8) and np.all(rates < 4.4), (errs, rates)


def test_periodic_translation_converges(orc):
    p, T = 2, 1.0
    vel = orc.Velocity("uniform", 1.0, 1.0)
    errs = []
    for n in (8, 16):
        pb = orc.Problem(dim=2, nx=n, ny=n, p=p, Gamma=0.0, eps=0.05)
        x, y = orc.tri_nodes(pb)
        f = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
        dt = 0.25 / (n * (2 * p + 1))
        ns = int(round(T / dt))
        w = orc.tri_rk4(pb, vel, np.stack([f, f]), 0.0, T / ns, ns)   # one period in x and y
        errs.append(np.abs(w[0] - f).max())
        assert np.abs(w[0] - w[1]).max() < 1e-12
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p), (errs, rates)


def test_rk4_fourth_order_with_a_time_dependent_velocity(orc):
    """Rider-Kothe velocity with period 0.5: pins the stage times t, t + dt/2, t + dt/2, t + dt."""
    pb = orc.Problem(dim=2, nx=3, ny=3, p=2, Gamma=0.5, eps=0.05, c_ip=2.0)
    vel = orc.Velocity("rider_kothe", T=0.5)
    x, y = orc.tri_nodes(pb)
    w0 = np.stack([0.5 + 0.4 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y), np.cos(2 * np.pi * (x + 0.3 * y))])
    T = 0.01
    sols = [orc.tri_rk4(pb, vel, w0, 0.1, T / n, n) for n in (16, 32, 64)]
    d1, d2 = np.abs(sols[0] - sols[1]).max(), np.abs(sols[1] - sols[2]).max()
    assert 12.0 < d1 / d2 < 20.0, (d1, d2, d1 / d2)
