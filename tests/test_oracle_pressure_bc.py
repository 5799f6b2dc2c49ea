"""Pins of the oracle's Riemann-invariant boundary "with zero velocity and constant pressure"
(Sec. 4.2, Rayleigh-Taylor and rising-bubble tests): the exterior state of the boundary
Riemann problem holds the own phase field and partial densities at rest at the prescribed
pressure P_b.  Checked against what the physics fixes:

* a state at rest at P = P_b is steady (the boundary exerts exactly the interior pressure);
* a hydrostatic column whose top pressure is P_b is steady;
* with the interior at rest at P != P_b, relative to a no-slip wall the boundary changes only the
  face nodes on it: no mass and no tangential momentum cross, and the normal momentum gains the
  pressure difference, M^-1 w_f (P - P_b) / 2 (the Lax-Friedrichs average of P and P_b in place
  of P), so the fluid is pushed out where P > P_b and drawn in where P < P_b.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import mass_weights, problem


def _box(bc, p_bc, g=0.0, n=(3, 4), p=3):
    return W.Workload(name="pb", dim=2, nx=n[0], ny=n[1], p=p, bc=bc, p_bc=p_bc, gamma=(1.4, 4.4),
                      pinf=(0.0, 6e8), rho0=(1.0, 1000.0), g=(0.0, g), gravity=g != 0.0, Gamma=0.0, eps=0.0)


def _rest_energy(wl, phi, P):
    """rho E of a state at rest at pressure P, written as the stiffened-gas relation
    P sum phi_l/(gamma_l - 1) + sum phi_l gamma_l Pinf_l/(gamma_l - 1)."""
    gi = [1.0 / (wl.gamma[l] - 1.0) for l in range(2)]
    C = [wl.gamma[l] * wl.pinf[l] / (wl.gamma[l] - 1.0) for l in range(2)]
    return P * (phi * gi[0] + (1.0 - phi) * gi[1]) + (phi * C[0] + (1.0 - phi) * C[1])


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_rest_state_at_boundary_pressure_is_steady(orc, side):
    bc = ["noslip"] * 4
    bc[side] = "pressure"
    pbc = [0.0] * 4
    pbc[side] = 2.5e5
    wl = _box(tuple(bc), tuple(pbc))
    w = np.array(W.conserved(wl, np.full(wl.N, 0.35), np.zeros(wl.N), 2.5e5, 0.0, 0.0))
    w[6] = _rest_energy(wl, w[0], 2.5e5)          # the exterior state's rho E, to the last bit
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    for v in range(7):
        assert np.abs(L[v]).max() <= 1e-13 * max(S[v].max(), 1.0), v


def test_hydrostatic_column_with_pressure_top_is_steady(orc):
    g = -9.81
    wl = _box(("slip", "slip", "noslip", "pressure"), (0.0, 0.0, 0.0, 1e5), g=g)
    x, y = W.node_coords(wl)
    P = 1e5 + 1000.0 * 0.6 * g * (y - wl.y1) + 1.0 * 0.4 * g * (y - wl.y1)
    w = W.conserved(wl, np.full(wl.N, 0.4), np.zeros(wl.N), P, 0.0, 0.0)
    rho = w[2] + w[3]
    assert np.allclose(rho, rho[0])
    P = 1e5 + rho[0] * g * (y - wl.y1)                 # exactly linear with dP/dy = rho g
    w = W.conserved(wl, np.full(wl.N, 0.4), np.zeros(wl.N), P, 0.0, 0.0)
    L, S = orc.rhs(problem(orc, wl), w, want_scale=True)
    assert np.abs(L[4]).max() < 1e-11 * S[4].max()
    assert np.abs(L[5]).max() < 1e-11 * S[5].max()


@pytest.mark.parametrize("Pb", [0.8e5, 1.3e5])
def test_pressure_difference_acts_on_the_boundary_nodes_only(orc, Pb):
    P0 = 1e5
    wa = _box(("noslip",) * 4, (0.0,) * 4)
    wb = _box(("noslip", "noslip", "noslip", "pressure"), (0.0, 0.0, 0.0, Pb))
    x, y = W.node_coords(wa)
    phi = 0.3 + 0.4 * (x - wa.x0) / (wa.x1 - wa.x0)
    w = W.conserved(wa, phi, np.zeros(wa.N), P0, 0.0, 0.0)
    La = orc.rhs(problem(orc, wa), w)
    Lb = orc.rhs(problem(orc, wb), w)
    d = Lb - La
    top = np.isclose(y, wb.y1)
    assert np.abs(d[[0, 2, 3, 4]]).max() < 1e-9 * np.abs(La[[2, 3, 4]]).max() + 1e-300
    assert np.all(np.abs(d[5][~top]) == 0.0) and np.all(np.abs(d[6][~top]) == 0.0)
    # M^-1 w_f at a north face node = (w_k h_x / 2) / (w_k w_p J) = 1 / (w_p h_y / 2)
    _, wt = orc.gll(wb.p)
    expected = 0.5 * (P0 - Pb) / (wt[-1] * 0.5 * wb.hy)
    # the stiffened-gas pressure recovery of both states carries ~1e-11 relative rounding
    assert np.allclose(d[5][top], expected, rtol=1e-10, atol=0)
    assert np.sign(d[5][top]).tolist() == [np.sign(P0 - Pb)] * int(top.sum())


def test_outflow_carries_half_the_interior_mass_flux(orc):
    """Uniform state moving towards the pressure boundary at v, at P = P_b, periodic in x with a
    no-slip bottom: the Lax-Friedrichs flux between the interior and the exterior state at rest
    moves (m v + 0)/2 per unit length across the top (the jump of m is zero), so the discrete
    mass of each phase changes at -m_l v L_x / 2; the no-slip bottom passes nothing."""
    v = 0.3
    wl = _box(("periodic", "periodic", "noslip", "pressure"), (0.0, 0.0, 0.0, 2e5))
    w = np.array(W.conserved(wl, np.full(wl.N, 0.35), np.zeros(wl.N), 2e5, 0.0, v))
    L = orc.rhs(problem(orc, wl), w)
    M = mass_weights(orc, wl)
    Lx = wl.x1 - wl.x0
    for l in (2, 3):
        assert np.isclose(np.sum(M * L[l]), -0.5 * w[l][0] * v * Lx, rtol=1e-12, atol=0), l
