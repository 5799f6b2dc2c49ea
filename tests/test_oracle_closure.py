"""Pins of the oracle's pointwise closure (Sec. 2: stiffened-gas EOS, sound speed,
phasic enthalpy, mixture rules) against textbook limits."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem


def _one_node_state(wl, phi, rho1, rho2, rhoe, u, v):
    n = wl.N
    m1 = rho1 * phi
    m2 = rho2 * (1 - phi)
    rho = m1 + m2
    w = np.zeros((7, n))
    w[0], w[2], w[3] = phi, m1, m2
    w[4], w[5] = rho * u, rho * v
    w[6] = rhoe + 0.5 * rho * (u * u + v * v)
    return w


@pytest.mark.parametrize("phase", [0, 1])
def test_pure_phase_is_textbook_stiffened_gas(orc, phase):
    """phi_l = 1: P = (gamma - 1) rho e - gamma Pinf, c^2 = gamma (P + Pinf)/rho."""
    wl = W.Workload(name="c", dim=1, nx=1, ny=1, p=1, gamma=(1.4, 4.4), pinf=(0.0, 6e8), rho0=(1.0, 1000.0))
    pb = problem(orc, wl)
    gam, pinf = wl.gamma[phase], wl.pinf[phase]
    rho = [1.2, 998.0][phase]
    rhoe = [2.5e5, 7.9e8][phase]
    phi = 1.0 if phase == 0 else 0.0
    w = _one_node_state(wl, phi, rho, rho, rhoe, 3.0, -2.0)
    prim = orc.primitives(pb, w)
    P_ref = (gam - 1.0) * rhoe - gam * pinf
    assert np.allclose(prim[3], P_ref, rtol=1e-12, atol=1e-9 * (gam * pinf + rhoe) * 1e-3)
    c_ref = np.sqrt(gam * (P_ref + pinf) / rho)
    np.testing.assert_allclose(prim[4], c_ref, rtol=1e-12)
    np.testing.assert_allclose(prim[0], rho, rtol=1e-15)


def test_enthalpy_difference_matches_internal_energy_form(orc):
    """B = rho_1 H_1 - rho_2 H_2 equals rho_1 h_1 - rho_2 h_2 with rho_l h_l = rho_l e_l + P,
    rho_l e_l = (P + gamma_l Pinf_l)/(gamma_l - 1): the two enthalpy forms agree."""
    wl = W.Workload(name="c", dim=1, nx=2, ny=1, p=2, gamma=(1.4, 4.4), pinf=(0.0, 6e8), rho0=(1.0, 1000.0))
    pb = problem(orc, wl)
    rng = np.random.default_rng(0)
    phi = rng.uniform(0, 1, wl.N)
    P = rng.uniform(5e4, 2e5, wl.N)
    w = W.conserved(wl, phi, np.zeros(wl.N), P, 1.5, 0.0)
    prim = orc.primitives(pb, w)
    Pp = prim[3]
    g, pi = wl.gamma, wl.pinf
    B_ref = (Pp + g[0] * pi[0]) / (g[0] - 1) + Pp - ((Pp + g[1] * pi[1]) / (g[1] - 1) + Pp)
    np.testing.assert_allclose(prim[5], B_ref, rtol=1e-12)
    np.testing.assert_allclose(Pp, P, rtol=1e-9)


def test_identical_phases_reduce_to_single_fluid(orc):
    """With identical phase constants the mixture is that fluid, whatever phi is."""
    wl = W.Workload(name="c", dim=1, nx=2, ny=1, p=2, gamma=(1.67, 1.67), pinf=(1e3, 1e3), rho0=(2.0, 2.0))
    pb = problem(orc, wl)
    rng = np.random.default_rng(1)
    phi = rng.uniform(0, 1, wl.N)
    rhoe = 3e4
    w = _one_node_state(wl, phi, 2.0, 2.0, rhoe, 0.5, 0.0)
    prim = orc.primitives(pb, w)
    P_ref = 0.67 * rhoe - 1.67 * 1e3
    np.testing.assert_allclose(prim[3], P_ref, rtol=1e-12)
    np.testing.assert_allclose(prim[4], np.sqrt(1.67 * (P_ref + 1e3) / 2.0), rtol=1e-12)
    np.testing.assert_allclose(prim[5], 0.0, atol=1e-9)
