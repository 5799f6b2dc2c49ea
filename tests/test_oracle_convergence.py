"""Convergence pins of the oracle (Sec. 4.1: the diffusion/sharpening terms must not
spoil the optimal order p + 1), the third-order SSP Runge-Kutta integrator, and the
FP64 diagnostics (integrals, Sec. 4.1.2 mass error)."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import mass_weights, problem

EPS = 0.0125


def _slab_fields(x):
    """Periodic slab of phase 2, |x - 0.5| < 0.25, with a signed distance psi growing into
    phase 1.  With eps = 0.0125 the kinks of psi sit where phi(1 - phi) < 1e-8."""
    s = np.abs(((x - 0.5 + 0.5) % 1.0) - 0.5) - 0.25
    return W.tanh_profile(s, EPS), s


def _translate(orc, n, p, T=0.05, dt=None):
    """Advect the slab at u = 1 with uniform P: the exact solution is a translation, since
    a_1 vanishes on the tanh profile.  Returns the L1 error of phi (as in Sec. 4.1)."""
    wl = W.Workload(name="cv", dim=1, nx=n, ny=1, p=p, gamma=(1.4, 1.6), pinf=(0.0, 0.0),
                    rho0=(1.0, 2.0), Gamma=1.0, eps=EPS)
    x, _ = W.node_coords(wl)
    phi, s = _slab_fields(x)
    w = W.conserved(wl, phi, s, 1.0, 1.0, 0.0)
    h = wl.hx
    q = 2 * p + 1
    if dt is None:
        dt = min(0.2 * h / (q * 2.3), 0.1 * h * h / (q * q * EPS))
    nst = int(np.ceil(T / dt))
    w = orc.rk3(problem(orc, wl), w, T / nst, nst)
    phie, _ = _slab_fields(x - T)
    return np.sum(mass_weights(orc, wl) * np.abs(w[0] - phie)), w


@pytest.mark.parametrize("p", [1, 2, 3])
def test_spatial_order_p_plus_one(orc, p):
    e1, _ = _translate(orc, 40, p)
    e2, _ = _translate(orc, 80, p)
    rate = np.log2(e1 / e2)
    assert rate > p + 0.7, (e1, e2, rate)


def test_ssp_rk3_is_third_order_in_time(orc):
    """Fixed mesh, smooth data, three time steps: successive differences shrink by 2^3."""
    wl = W.Workload(name="t", dim=1, nx=10, ny=1, p=3, gamma=(1.4, 1.6), pinf=(0.0, 0.0),
                    rho0=(1.0, 2.0), Gamma=0.5, eps=0.05)
    x, _ = W.node_coords(wl)
    phi = 0.5 + 0.3 * np.sin(2 * np.pi * x)
    psi = np.sin(2 * np.pi * x)
    P = 1.0 + 0.1 * np.cos(2 * np.pi * x)
    u = 0.5 + 0.2 * np.sin(4 * np.pi * x)
    w0 = W.conserved(wl, phi, psi, P, u, 0.0)
    pb = problem(orc, wl)
    T = 0.02  # stable for dt <= ~8e-4 (parabolic limit of the SIP term)
    sols = [orc.rk3(pb, w0, T / n, n) for n in (32, 64, 128)]
    d1 = np.abs(sols[0] - sols[1]).max()
    d2 = np.abs(sols[1] - sols[2]).max()
    assert 6.5 < d1 / d2 < 9.5, d1 / d2


def test_diag_integrals_and_extrema(orc):
    """Integrals are GLL quadrature sums, exact for polynomials of degree <= 2p - 1."""
    wl = W.Workload(name="d", dim=2, nx=3, ny=2, p=3, x0=0, x1=2, y0=-1, y1=1)
    x, y = W.node_coords(wl)
    phi = 0.2 + 0.1 * x * y ** 2         # exact integral over [0,2]x[-1,1]: 0.8 + 0.1*2*(2/3) = 0.9333..
    w = W.conserved(wl, phi, x ** 3, 1e5, 0.0, 0.0)
    d = orc.diag(problem(orc, wl), w)
    assert abs(d[0] - (0.8 + 0.4 / 3.0)) < 1e-14
    assert abs(d[1] - 8.0) < 1e-13          # int x^3 = 2^4/4 * 2
    assert d[7] == pytest.approx(phi.min(), abs=0) and d[8] == pytest.approx(phi.max(), abs=0)
    assert d[15] == 0
