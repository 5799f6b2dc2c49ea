"""Pins of the oracle's BR1-lifted gradient option (grad_lift): the gradients of phi and psi taken
as the broken gradient plus the lifting of the face jumps with central traces,
    q = grad_h f + M^-1 sum_faces int l ({f} - f-) m,
which the scheme then uses for a_1, the level-set normal, the SIP flux's {grad phi} and the CSF
delta (Sec. 3 leaves the gradient discretisation open; the broken gradient is the default).

* on fields continuous across faces the lifting adds exactly nothing;
* the lifted gradient of any nodal field on a periodic mesh integrates to zero (the gradient of a
  periodic function, jumps included), which the broken gradient does not;
* for a field constant on every element it is (f+ - f-) / (w_0 h) m at the face nodes and zero
  elsewhere (w_0 the GLL end weight);
* the interface equilibrium and the conservation of the scheme hold with it, and the planar tanh
  profile stays an equilibrium.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import mass_weights, problem


def _lifted(wl):
    wl2 = W.Workload(**{k: getattr(wl, k) for k in wl.problem_kwargs()}, name=wl.name)
    wl2.grad_lift = True
    wl2.w = wl.w
    return wl2


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (2, 4), (1, 3)])
def test_lifting_adds_nothing_to_continuous_fields(orc, dim, p):
    wl = W.Workload(name="c", dim=dim, nx=4, ny=4 if dim == 2 else 1, p=p, Gamma=0.8, eps=0.05)
    x, y = W.node_coords(wl)
    f = np.sin(2 * np.pi * x) * (np.cos(2 * np.pi * y) if dim == 2 else 1.0) + 0.3
    gb = orc.gradients(problem(orc, wl), f)
    gl = orc.gradients(problem(orc, _lifted(wl)), f)
    # (at the periodic seam the field is continuous up to the rounding of its evaluation)
    for d in range(2):
        assert np.abs(gl[d] - gb[d]).max() <= 1e-12 * np.abs(gb[0]).max(), d
    # and the whole right-hand side of a state continuous across faces is unchanged
    if dim == 2:
        s = W.periodic_distance(x, y, 0.4, 0.55) - 0.2
        w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, 0.7, -0.2)
        L0, S = orc.rhs(problem(orc, wl), w, want_scale=True)
        L1 = orc.rhs(problem(orc, _lifted(wl)), w)
        for v in range(7):
            assert np.abs(L1[v] - L0[v]).max() <= 1e-12 * S[v].max(), v


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (1, 4)])
def test_lifted_gradient_integrates_to_zero_on_a_periodic_mesh(orc, dim, p):
    wl = W.Workload(name="r", dim=dim, nx=5, ny=3 if dim == 2 else 1, p=p)
    rng = np.random.default_rng(3)
    f = rng.normal(size=wl.N)  # jumps at every face
    M = mass_weights(orc, wl)
    gl = orc.gradients(problem(orc, _lifted(wl)), f)
    gb = orc.gradients(problem(orc, wl), f)
    scale = np.sum(M * np.abs(gb[0]))
    for d in range(dim):
        assert abs(np.sum(M * gl[d])) < 1e-13 * scale, d
    assert abs(np.sum(M * gb[0])) > 1e-3 * scale  # the broken gradient does not


@pytest.mark.parametrize("dim,p", [(2, 3), (2, 4), (1, 2)])
def test_lifted_gradient_of_piecewise_constant_field(orc, dim, p):
    """f = c_e on element e: the broken gradient vanishes, and the lifting puts (c_nb - c_e) / (w_0 h)
    times the outward normal at each face node (two such terms at a corner)."""
    wl = W.Workload(name="pc", dim=dim, nx=4, ny=3 if dim == 2 else 1, p=p, x1=1.2, y1=0.9)
    rng = np.random.default_rng(5)
    ce = rng.normal(size=wl.E)
    f = np.repeat(ce, wl.Np)
    gx, gy = orc.gradients(problem(orc, _lifted(wl)), f)
    _, wt = orc.gll(p)
    P1 = p + 1
    ex_of = lambda e: e % wl.nx
    ey_of = lambda e: e // wl.nx
    ref_x, ref_y = np.zeros(wl.N), np.zeros(wl.N)
    for e in range(wl.E):
        ex, ey = ex_of(e), ey_of(e)
        west = ey * wl.nx + (ex - 1) % wl.nx
        east = ey * wl.nx + (ex + 1) % wl.nx
        for a in range(wl.Np):
            i, j = a % P1, (a // P1 if dim == 2 else 0)
            n = e * wl.Np + a
            if i == 0:
                ref_x[n] += -(ce[west] - ce[e]) / (wt[0] * wl.hx)
            if i == p:
                ref_x[n] += (ce[east] - ce[e]) / (wt[0] * wl.hx)
            if dim == 2:
                south = ((ey - 1) % wl.ny) * wl.nx + ex
                north = ((ey + 1) % wl.ny) * wl.nx + ex
                if j == 0:
                    ref_y[n] += -(ce[south] - ce[e]) / (wt[0] * wl.hy)
                if j == p:
                    ref_y[n] += (ce[north] - ce[e]) / (wt[0] * wl.hy)
    np.testing.assert_allclose(gx, ref_x, rtol=1e-13, atol=1e-13 * np.abs(ref_x).max())
    if dim == 2:
        np.testing.assert_allclose(gy, ref_y, rtol=1e-13, atol=1e-13 * np.abs(ref_y).max())


def test_no_lifting_through_walls(orc):
    """At walls the exterior value is the own one: a global polynomial of degree <= p on a box with
    walls keeps its exact gradient (no jumps anywhere)."""
    p = 3
    wl = W.Workload(name="box", dim=2, nx=3, ny=3, p=p, bc=("noslip", "slip", "noslip", "slip"),
                    x0=-1, x1=1, y0=-1, y1=1, grad_lift=True)
    x, y = W.node_coords(wl)
    f = 0.3 * x ** 3 - x * y ** 2 + 0.5 * y ** 3 - y
    gx, gy = orc.gradients(problem(orc, wl), f)
    np.testing.assert_allclose(gx, 0.9 * x ** 2 - y ** 2, atol=1e-12)
    np.testing.assert_allclose(gy, -2 * x * y + 1.5 * y ** 2 - 1, atol=1e-12)


def _broken_state(wl, seed=11, amp=0.05):
    rng = np.random.default_rng(seed)
    x, y = W.node_coords(wl)
    s = W.periodic_distance(x, y, 0.45, 0.5) - 0.22
    phi = np.clip(W.tanh_profile(s, wl.eps) + amp * rng.uniform(-1, 1, wl.N), 0.0, 1.0)
    psi = s + amp * rng.uniform(-1, 1, wl.N)
    return phi, psi


def test_interface_equilibrium_with_lifted_gradients(orc):
    """Uniform u and P with a phase field and level set that jump at every face: the a_1-derived
    terms stay the phi-equation flux times the face coefficients, so rho u and P stay uniform."""
    wl = W.drop_2d(n=5, p=3, seed=2)
    wl.grad_lift = True
    phi, psi = _broken_state(wl)
    w = W.conserved(wl, phi, psi, 1e5, 1.0, 0.5)
    pb = problem(orc, wl)
    L, S = orc.rhs(pb, w, want_scale=True)
    prim = orc.primitives(pb, w)
    u, v, B = prim[1], prim[2], prim[5]
    Lrho = L[2] + L[3]
    k = 0.5 * (u * u + v * v)
    assert np.abs(L[4] - u * Lrho).max() < 1e-12 * S[4].max()
    assert np.abs(L[5] - v * Lrho).max() < 1e-12 * S[5].max()
    assert np.abs(L[6] - (B * L[0] + k * Lrho)).max() < 1e-12 * S[6].max()
    # and the lifting changes the phase-field rate of this state (the option is in effect)
    wl0 = W.drop_2d(n=5, p=3, seed=2)
    L0 = orc.rhs(problem(orc, wl0), w)
    assert np.abs(L[0] - L0[0]).max() > 1e-6 * S[0].max()


def test_conservation_with_lifted_gradients(orc):
    wl = W.drop_2d(n=5, p=3, seed=2)
    wl.grad_lift = True
    phi, psi = _broken_state(wl)
    x, y = W.node_coords(wl)
    w = W.conserved(wl, phi, psi, 1e5 * (1 + 0.01 * np.sin(2 * np.pi * x)), 0.6 + 0.2 * np.cos(2 * np.pi * y), -0.3)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    M = mass_weights(orc, wl)
    for var in (2, 3, 4, 5, 6):
        assert abs(np.sum(M * L[var])) < 1e-13 * np.sum(M * S[var]), var


@pytest.mark.parametrize("p", [3, 4])
def test_planar_tanh_equilibrium_with_lifted_gradients(orc, p):
    """u = 0, phi = tanh profile of s, psi = s (walls all round): a_1 vanishes analytically, so L(phi)
    is discretisation error and shrinks under refinement with the lifted gradients too."""
    errs = []
    for n in (10, 20, 40):
        wl = W.Workload(name="pl", dim=2, nx=n, ny=n, p=p, bc=("noslip",) * 4, Gamma=1.0, eps=0.05,
                        grad_lift=True)
        x, y = W.node_coords(wl)
        s = (x - 0.5) * np.cos(0.3) + (y - 0.5) * np.sin(0.3)
        w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, 0.0, 0.0)
        errs.append(np.abs(orc.rhs(problem(orc, wl), w)[0]).max())
    assert errs[-1] < 0.03
    assert np.log2(errs[1] / errs[2]) > 1.5
