"""The rising-bubble workload against the paper's statement of the test (Sec. 4.2, "Rising
bubble"): geometry, boundary kinds, the density and viscosity ratios and the Reynolds and Eotvos
numbers of both cases, and a hydrostatic initial pressure."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W


@pytest.mark.parametrize("case,ratios,Eo", [(1, (10.0, 10.0), 10.0), (2, (1000.0, 100.0), 125.0)])
def test_rising_bubble_numbers(case, ratios, Eo):
    wl = W.rising_bubble(nx=20, ny=40, p=2, case=case)
    (rho1, rho2), (mu1, mu2) = wl.rho0, wl.mu
    g, R = abs(wl.g[1]), 0.25
    assert (wl.x0, wl.x1, wl.y0, wl.y1) == (-0.5, 0.5, 0.0, 2.0)
    assert wl.bc == ("slip", "slip", "noslip", "pressure") and wl.g[0] == 0.0 and wl.g[1] < 0.0
    assert rho1 / rho2 == pytest.approx(ratios[0]) and mu1 / mu2 == pytest.approx(ratios[1])
    assert rho1 * (2 * R) ** 1.5 * np.sqrt(g) / mu1 == pytest.approx(35.0)      # Re
    assert 4 * rho1 * g * R * R / wl.sigma == pytest.approx(Eo)                # Eo
    # the bubble (phase 2, phi -> 0) at (0, 0.5) with radius 0.25, the heavy phase 1 around it
    x, y = W.node_coords(wl)
    r = np.hypot(x, y - 0.5)
    assert np.all(wl.w[0][r < 0.1] < 0.05) and np.all(wl.w[0][r > 0.5] > 0.95)
    assert np.allclose(wl.w[1], r - R)


def test_rising_bubble_pressure_is_hydrostatic():
    """Far from the bubble the initial pressure is P_top + rho_1 |g| (2 - y); above the bubble the
    column holds less heavy fluid by (rho_1 - rho_2) |g| times the bubble's chord."""
    wl = W.rising_bubble(nx=10, ny=20, p=3)
    x, y = W.node_coords(wl)
    rho1, rho2 = wl.rho0
    g = abs(wl.g[1])
    phi = wl.w[0]
    rho = wl.w[2] + wl.w[3]
    P = (wl.w[6] - 0.5 * (wl.w[4] ** 2 + wl.w[5] ** 2) / rho - (phi * 4.4 * 6e8 / 3.4 + (1 - phi) * 4.4 * 6e8 / 3.4)) \
        / (phi / 3.4 + (1 - phi) / 3.4)
    far = (np.abs(x) > 0.45) & (y > 1.3)
    assert np.allclose(P[far], 1e5 + rho1 * g * (2.0 - y[far]), rtol=0, atol=1e-3 * rho1 * g)
    # at the bottom below the centre: the column crosses the whole bubble, chord 2R
    below = (np.abs(x) < 1e-12) & (y < 1e-12)
    assert below.any()
    expect = 1e5 + rho1 * g * 2.0 - (rho1 - rho2) * g * 0.5
    assert np.allclose(P[below], expect, rtol=0, atol=0.02 * (rho1 - rho2) * g * 0.5)
