"""Pins of the oracle's level-set re-initialisation (end of Sec. 3):
    d(psi)/d(tau) = S (1 - |grad psi|) + div(nu grad psi),  psi(0) = psi0 = phi - 1/2,
    S = tanh(psi0 / (2 eps |grad psi0|)),
checked against what the mathematics fixes:

* on the tanh profile phi = (1 + tanh(s / 2 eps)) / 2 the smeared sign has the closed form
  S = tanh(sinh(s / eps) / 2) (psi0 / (2 eps |grad psi0|) = sinh(s/2eps) cosh(s/2eps));
* with nu = 0 the right-hand side is the nodal source S (1 - |grad psi|), exact for a level set
  that the basis represents exactly (a quadratic);
* with S = 0 it is the SIP diffusion alone: M L symmetric, negative semi-definite, constants in
  its null space;
* on a planar slab the iteration relaxes |grad psi| towards 1 near the interface and keeps the
  zero level set in place (with the hyperbolic term's sign as printed, |grad psi| would grow).
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W


def _weights(orc, pb):
    _, wt = orc.gll(pb.p)
    hx, hy = (pb.x1 - pb.x0) / pb.nx, (pb.y1 - pb.y0) / pb.ny
    return np.tile(np.outer(wt, wt).ravel() * 0.25 * hx * hy, pb.nx * pb.ny)


def _grad_norm(orc, pb, psi):
    """|grad psi| at the nodes: with S = -1 and nu = 0 the right-hand side is |grad psi| - 1."""
    return 1.0 + orc.reinit_rhs(pb, -np.ones(pb.N), psi, 0.0)


def test_smeared_sign_closed_form_on_tanh_profile(orc):
    eps = 0.05
    pb = orc.Problem(dim=2, nx=80, ny=1, p=4, Gamma=1.0, eps=eps)
    x, _ = orc.nodes(pb)
    s = x - 0.5
    S = orc.reinit_sign(pb, W.tanh_profile(s, eps))
    near = np.abs(s) < 3 * eps
    assert np.abs(S[near] - np.tanh(0.5 * np.sinh(s[near] / eps))).max() < 2e-3
    assert np.all(np.abs(S) <= 1.0) and np.all(np.sign(S[np.abs(s) > 1e-9]) == np.sign(s[np.abs(s) > 1e-9]))


@pytest.mark.parametrize("p", [2, 3])
def test_source_is_exact_for_a_quadratic_level_set(orc, p):
    pb = orc.Problem(dim=2, nx=3, ny=4, p=p, Gamma=1.0, eps=0.05)
    x, y = orc.nodes(pb)
    psi = 0.3 * x * x - 0.2 * x * y + 0.5 * y + 0.1
    gx, gy = 0.6 * x - 0.2 * y, -0.2 * x + 0.5
    S = np.random.default_rng(p).uniform(-1, 1, pb.N)
    L = orc.reinit_rhs(pb, S, psi, 0.0)
    assert np.abs(L - S * (1.0 - np.hypot(gx, gy))).max() < 1e-13


@pytest.mark.parametrize("p,n,bc", [(1, 4, "periodic"), (2, 3, "periodic"), (3, 2, "noslip")])
def test_diffusion_operator_symmetric_negative_semidefinite(orc, p, n, bc):
    pb = orc.Problem(dim=2, nx=n, ny=n, p=p, bc=(bc,) * 4, Gamma=1.0, eps=0.05)
    N = pb.N
    M = _weights(orc, pb)
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = M * orc.reinit_rhs(pb, np.zeros(N), e, 0.3)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-12 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-11 * scale
    assert np.abs(A @ np.ones(N)).max() <= 1e-12 * scale


def test_planar_slab_relaxes_to_unit_gradient_in_place(orc):
    eps, p, n = 0.04, 3, 24
    pb = orc.Problem(dim=2, nx=n, ny=1, p=p, Gamma=1.0, eps=eps)
    x, _ = orc.nodes(pb)
    s = 0.25 - np.abs(x - 0.5)                       # slab of phase 1, |x - 0.5| < 0.25
    phi = W.tanh_profile(s, eps)
    h, q = 1.0 / n, 2 * p + 1
    nu = 0.5 * h / (p + 1)
    dtau = min(0.5 * h / q, 0.1 * h * h / (q * q * nu))
    band = np.abs(s) < eps
    dev = []
    for nit in (0, 50, 100, 200):
        psi = orc.reinit(pb, phi, nit, nu, dtau)
        dev.append(np.abs(_grad_norm(orc, pb, psi)[band] - 1.0).max())
        keep = np.abs(s) > 0.2 * eps
        assert np.all(np.sign(psi[keep & band]) == np.sign(s[keep & band])), nit
    assert all(b < a for a, b in zip(dev, dev[1:])), dev
    assert dev[-1] < 0.25 * dev[0], dev
