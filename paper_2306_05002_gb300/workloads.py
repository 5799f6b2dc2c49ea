"""Seeded synthetic workloads shaped like the paper's test cases (Sec. 4).

This module is shared by the tests and the benchmark; it holds none of the
DG method's arithmetic.  It only

* places analytic initial conditions at Gauss-Lobatto-Legendre points (found
  with ``numpy.polynomial.legendre``), in the state layout of the library,
* writes them in conserved form by solving the stiffened-gas relation of
  Sec. 2 for the internal energy, rho e = P sum phi_l/(gamma_l-1) +
  sum phi_l gamma_l Pinf_l/(gamma_l-1), and
* picks a time step from the pure-phase sound speeds and a CFL number.

Phase 1 is the outer (or upper) phase and phi = phi_1 its volume fraction.
The interface profile is phi = (1 + tanh(s / (2 eps))) / 2 with s a signed
distance that grows into phase 1, and the level set is psi = s (Sec. 4.1;
the sign of psi is chosen so that n = grad psi/|grad psi| points into phase 1,
which makes the hyperbolic-tangent profile an equilibrium of a_1).

Nothing here is drawn from a dataset: every field is analytic, and every
random number comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

AIR = dict(gamma=1.4, pinf=0.0, rho0=1.0)
WATER = dict(gamma=4.4, pinf=6e8, rho0=1000.0)


@dataclass
class Workload:
    """A DG problem plus its initial state, time step and step count."""
    name: str
    dim: int
    nx: int
    ny: int
    p: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    bc: tuple = ("periodic",) * 4
    gamma: tuple = (1.4, 4.4)
    pinf: tuple = (0.0, 6e8)
    rho0: tuple = (1.0, 1000.0)
    mu: tuple = (0.0, 0.0)
    sigma: float = 0.0
    g: tuple = (0.0, 0.0)
    Gamma: float = 1.0
    eps: float = 0.01
    c_ip: float = 1.0
    viscous: bool = False
    gravity: bool = False
    surface_tension: bool = False
    p_bc: tuple = (0.0, 0.0, 0.0, 0.0)  # exterior pressure of "pressure" sides
    grad_lift: bool = False            # BR1-lifted gradients of phi and psi
    w: Optional[np.ndarray] = None   # (7, N) float64
    dt: float = 0.0
    nsteps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def Np(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def E(self) -> int:
        return self.nx * self.ny

    @property
    def N(self) -> int:
        return self.E * self.Np

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self) -> float:
        return (self.y1 - self.y0) / self.ny if self.dim == 2 else self.hx

    def problem_kwargs(self) -> dict:
        """Fields shared by the oracle's and the library's problem descriptions."""
        keys = ["dim", "nx", "ny", "p", "x0", "x1", "y0", "y1", "bc", "gamma", "pinf", "rho0", "mu",
                "sigma", "g", "Gamma", "eps", "c_ip", "viscous", "gravity", "surface_tension", "p_bc", "grad_lift"]
        return {k: getattr(self, k) for k in keys}


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

def gll_points(p: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre points on [-1, 1]: the end points and the roots of P_p'."""
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def node_coords(wl: Workload):
    """x, y of every node in the state layout: node n = e * Np + i + (p+1) j, e = ex + nx ey."""
    xi = gll_points(wl.p)
    P1 = wl.p + 1
    ex = np.arange(wl.nx)
    if wl.dim == 1:
        x = wl.x0 + wl.hx * (ex[:, None] + 0.5 * (xi[None, :] + 1.0))
        return x.reshape(-1), np.zeros(wl.N)
    ey = np.arange(wl.ny)
    # shape (ny, nx, P1[j], P1[i])
    x = wl.x0 + wl.hx * (ex[None, :, None, None] + 0.5 * (xi[None, None, None, :] + 1.0))
    y = wl.y0 + wl.hy * (ey[:, None, None, None] + 0.5 * (xi[None, None, :, None] + 1.0))
    x = np.broadcast_to(x, (wl.ny, wl.nx, P1, P1))
    y = np.broadcast_to(y, (wl.ny, wl.nx, P1, P1))
    return np.ascontiguousarray(x).reshape(-1), np.ascontiguousarray(y).reshape(-1)


# ---------------------------------------------------------------------------
# Conserved state from primitive fields
# ---------------------------------------------------------------------------

def conserved(wl: Workload, phi, psi, P, u, v, rho1=None, rho2=None) -> np.ndarray:
    """Pack phi, psi, m1, m2, rho u, rho v, rho E (rho_l defaults to the reference densities)."""
    g1, g2 = wl.gamma
    pi1, pi2 = wl.pinf
    rho1 = wl.rho0[0] if rho1 is None else rho1
    rho2 = wl.rho0[1] if rho2 is None else rho2
    phi2 = 1.0 - phi
    m1 = rho1 * phi
    m2 = rho2 * phi2
    rho = m1 + m2
    rhoe = P * (phi / (g1 - 1.0) + phi2 / (g2 - 1.0)) + (phi * g1 * pi1 / (g1 - 1.0) + phi2 * g2 * pi2 / (g2 - 1.0))
    rhoE = rhoe + 0.5 * rho * (u * u + v * v)
    w = np.stack([phi, psi, m1, m2, rho * u, rho * v, rhoE]).astype(np.float64)
    return np.ascontiguousarray(np.broadcast_to(w, (7, wl.N)))


def tanh_profile(s, eps):
    return 0.5 * (1.0 + np.tanh(s / (2.0 * eps)))


def stable_dt(wl: Workload, umax: float, P0: float, cfl: float = 0.5) -> float:
    """CFL time step from the pure-phase sound speeds c_l = sqrt(gamma_l (P + Pinf_l)/rho_l).

    The acoustic limit cfl h / ((2p+1)(|u| + c)) holds for p <= 4; at p = 5 it sits at the edge
    of SSP-RK3's stability region for this scheme (at that step most order-5 drops and bubbles of
    the batched ensemble grow grid-scale oscillations and overflow within 200 steps, in FP64 as
    in FP32), so order 5 takes 0.9 of it."""
    c = max(np.sqrt(wl.gamma[l] * (P0 + wl.pinf[l]) / wl.rho0[l]) for l in range(2))
    h = min(wl.hx, wl.hy)
    q = 2 * wl.p + 1
    if wl.p >= 5:
        cfl *= 0.9
    dt = cfl * h / (q * (umax + c))
    # the interior-penalty diffusion operators need a tighter, parabolic limit
    if wl.Gamma * wl.eps > 0:
        dt = min(dt, 0.1 * h * h / (q * q * wl.Gamma * wl.eps))
    if wl.viscous and max(wl.mu) > 0:
        nu = max(wl.mu) / min(wl.rho0)
        dt = min(dt, 0.1 * h * h / (q * q * nu))
    return dt


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def slab_1d(nx: int = 100, p: int = 3, nsteps: int = 1000, u: float = 1.0, P0: float = 1e5) -> Workload:
    """1D periodic advection of a water slab |x - 0.5| < 0.25 in air, eps = one element width."""
    wl = Workload(name=f"slab1d_{nx}p{p}", dim=1, nx=nx, ny=1, p=p, bc=("periodic",) * 4,
                  gamma=(AIR["gamma"], WATER["gamma"]), pinf=(AIR["pinf"], WATER["pinf"]),
                  rho0=(AIR["rho0"], WATER["rho0"]), nsteps=nsteps)
    wl.eps = wl.hx
    wl.Gamma = abs(u)
    x, _ = node_coords(wl)
    s = np.abs(x - 0.5) - 0.25          # grows into the air (phase 1)
    phi = tanh_profile(s, wl.eps)
    wl.w = conserved(wl, phi, s, P0, u, 0.0)
    wl.dt = stable_dt(wl, abs(u), P0)
    wl.meta = dict(P0=P0, u=u, v=0.0)
    return wl


def periodic_distance(x, y, cx, cy):
    dx = x - cx
    dy = y - cy
    dx -= np.round(dx)
    dy -= np.round(dy)
    return np.sqrt(dx * dx + dy * dy)


def drop_2d(n: int = 64, p: int = 3, seed: int = 2, R: float = 0.15, u: float = 1.0, v: float = 0.5,
            P0: float = 1e5, eps_h: float = 0.75, nsteps: int = 500, center=None,
            water_inside: bool = True) -> Workload:
    """Periodic unit square, water drop (or air bubble) of radius R at a seeded random centre."""
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0.0, 1.0, size=2) if center is None else center
    wl = Workload(name=f"drop2d_{n}x{n}p{p}", dim=2, nx=n, ny=n, p=p, bc=("periodic",) * 4,
                  gamma=(AIR["gamma"], WATER["gamma"]), pinf=(AIR["pinf"], WATER["pinf"]),
                  rho0=(AIR["rho0"], WATER["rho0"]), nsteps=nsteps)
    if not water_inside:  # air bubble in water: phase 1 (outer) is water
        wl.gamma, wl.pinf, wl.rho0 = wl.gamma[::-1], wl.pinf[::-1], wl.rho0[::-1]
    wl.eps = eps_h * wl.hx
    wl.Gamma = float(np.hypot(u, v))
    x, y = node_coords(wl)
    s = periodic_distance(x, y, cx, cy) - R
    phi = tanh_profile(s, wl.eps)
    wl.w = conserved(wl, phi, s, P0, u, v)
    wl.dt = stable_dt(wl, float(np.hypot(u, v)), P0)
    wl.meta = dict(P0=P0, u=u, v=v, cx=float(cx), cy=float(cy), R=R, seed=seed)
    return wl


def rayleigh_taylor(n: int = 256, p: int = 4, seed: int = 3, nsteps: int = 2000, P_top: float = 1e5,
                    eps_h: float = 0.75, Gamma: float = 2.21, amp: float = 0.01, modes: int = 8) -> Workload:
    """Viscous Rayleigh-Taylor set-up: heavy phase 1 on top, density ratio 3, no-slip walls,
    gravity -9.81, surface tension 0.07, hydrostatic pressure, seeded 8-mode interface."""
    rng = np.random.default_rng(seed)
    a = rng.normal(size=modes)
    a /= np.abs(a).sum()
    theta = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    g = 9.81
    rho1, rho2 = 3000.0, 1000.0
    mu = rho1 * np.sqrt(g) / 3000.0
    wl = Workload(name=f"rt2d_{n}x{n}p{p}", dim=2, nx=n, ny=n, p=p, bc=("noslip",) * 4,
                  gamma=(4.4, 4.4), pinf=(6e8, 6e8), rho0=(rho1, rho2), mu=(mu, mu), sigma=0.07,
                  g=(0.0, -g), Gamma=Gamma, viscous=True, gravity=True, surface_tension=True,
                  nsteps=nsteps)
    wl.eps = eps_h * wl.hx
    x, y = node_coords(wl)
    k = np.arange(1, modes + 1)
    eta = 0.5 + amp * np.sum(a[None, :] * np.cos(2 * np.pi * k[None, :] * x[:, None] + theta[None, :]), axis=1)
    s = y - eta                          # grows into the heavy upper phase 1
    phi = tanh_profile(s, wl.eps)
    # hydrostatic pressure P(y) = P_top + g int_y^1 rho(y') dy' with rho = rho2 + (rho1-rho2) phi
    def F(yy):  # antiderivative of phi along y: y/2 + eps log cosh((y - eta)/(2 eps))
        z = (yy - eta) / (2.0 * wl.eps)
        az = np.abs(z)
        return 0.5 * yy + wl.eps * (az + np.log1p(np.exp(-2.0 * az)) - np.log(2.0))
    P = P_top + g * (rho2 * (1.0 - y) + (rho1 - rho2) * (F(1.0) - F(y)))
    wl.w = conserved(wl, phi, s, P, 0.0, 0.0)
    wl.dt = stable_dt(wl, 0.0, P_top)
    wl.meta = dict(P_top=P_top, a=a.tolist(), theta=theta.tolist(), seed=seed)
    return wl


def rayleigh_taylor_paper(nx: int = 10, ny: int = 40, p: int = 4, P_top: float = 1e5, eps_h: float = 0.75,
                          Gamma: float = 2.21, Re: float = 3000.0) -> Workload:
    """The paper's Rayleigh-Taylor domain (Sec. 4.2): [0, d] x [0, 4d], d = 1, interface
    y = 2 + 0.1 cos(2 pi x), Atwood 0.5 (density ratio 3, heavy phase 1 on top), Re = 3000,
    gravity -9.81; no-slip bottom, slip sides, and the Riemann-invariant top boundary at rest at
    the hydrostatic top pressure.  Liquid-liquid closure as in `rayleigh_taylor`; no surface
    tension (the paper names none for this test)."""
    g = 9.81
    rho1, rho2 = 3000.0, 1000.0
    mu = rho1 * np.sqrt(g) / Re
    wl = Workload(name=f"rtp2d_{nx}x{ny}p{p}", dim=2, nx=nx, ny=ny, p=p, x0=0.0, x1=1.0, y0=0.0, y1=4.0,
                  bc=("slip", "slip", "noslip", "pressure"), p_bc=(0.0, 0.0, 0.0, P_top),
                  gamma=(4.4, 4.4), pinf=(6e8, 6e8), rho0=(rho1, rho2), mu=(mu, mu), g=(0.0, -g),
                  Gamma=Gamma, viscous=True, gravity=True)
    wl.eps = eps_h * min(wl.hx, wl.hy)
    x, y = node_coords(wl)
    s = y - (2.0 + 0.1 * np.cos(2 * np.pi * x))   # grows into the heavy upper phase 1
    phi = tanh_profile(s, wl.eps)
    eta = 2.0 + 0.1 * np.cos(2 * np.pi * x)
    def F(yy):  # antiderivative of phi along y
        z = (yy - eta) / (2.0 * wl.eps)
        az = np.abs(z)
        return 0.5 * yy + wl.eps * (az + np.log1p(np.exp(-2.0 * az)) - np.log(2.0))
    P = P_top + g * (rho2 * (4.0 - y) + (rho1 - rho2) * (F(4.0) - F(y)))
    wl.w = conserved(wl, phi, s, P, 0.0, 0.0)
    wl.dt = stable_dt(wl, 0.0, P_top)
    wl.meta = dict(P_top=P_top)
    return wl


def _trapezoid(f, x):
    """Trapezoidal rule along the last axis (numpy's name for it changed between versions)."""
    return np.sum(0.5 * (f[..., 1:] + f[..., :-1]) * np.diff(x, axis=-1), axis=-1)


def rising_bubble(nx: int = 10, ny: int = 20, p: int = 4, case: int = 1, P_top: float = 1e5,
                  eps_h: float = 0.75, nquad: int = 4000) -> Workload:
    """The paper's rising bubble (Sec. 4.2): a circular bubble of the light phase 2, radius
    R = 0.25, centred at (0, 0.5) in [-0.5, 0.5] x [0, 2], rising in the heavy phase 1 under
    gravity; no-slip bottom, slip sides and the Riemann-invariant top boundary at rest at P_top.
    Case 1: rho_1/rho_2 = mu_1/mu_2 = 10, Eo = 4 rho_1 |g| R^2 / sigma = 10; case 2:
    rho_1/rho_2 = 1000, mu_1/mu_2 = 100, Eo = 125; both Re = rho_1 d^(3/2) |g|^(1/2) / mu_1 = 35 with
    d = 2R.  rho_1 = 1000 and |g| = 0.98 fix the dimensional values (the paper states only the
    ratios and the numbers).  Liquid-liquid closure as in `rayleigh_taylor` (both phases gamma =
    4.4, Pinf = 6e8); Gamma = sqrt(|g| d / 2), the rule that gives `rayleigh_taylor`'s 2.21;
    eps = 0.75 h.  The pressure is hydrostatic: P_top plus |g| times the column integral of the
    density above each node (trapezoidal rule with `nquad` points)."""
    g, R, d = 0.98, 0.25, 0.5
    rho1 = 1000.0
    rho2, mu_ratio, Eo = (rho1 / 10.0, 10.0, 10.0) if case == 1 else (rho1 / 1000.0, 100.0, 125.0)
    mu1 = rho1 * d ** 1.5 * np.sqrt(g) / 35.0
    sigma = 4.0 * rho1 * g * R * R / Eo
    wl = Workload(name=f"rb{case}_{nx}x{ny}p{p}", dim=2, nx=nx, ny=ny, p=p, x0=-0.5, x1=0.5, y0=0.0, y1=2.0,
                  bc=("slip", "slip", "noslip", "pressure"), p_bc=(0.0, 0.0, 0.0, P_top),
                  gamma=(4.4, 4.4), pinf=(6e8, 6e8), rho0=(rho1, rho2), mu=(mu1, mu1 / mu_ratio),
                  sigma=sigma, g=(0.0, -g), Gamma=float(np.sqrt(g * d / 2.0)), viscous=True, gravity=True,
                  surface_tension=True)
    wl.eps = eps_h * min(wl.hx, wl.hy)
    x, y = node_coords(wl)
    s = np.hypot(x, y - 0.5) - R                  # grows into the heavy outer phase 1
    phi = tanh_profile(s, wl.eps)
    # hydrostatic pressure: P(x, y) = P_top + g int_y^2 rho(x, y') dy', rho = rho2 + (rho1 - rho2) phi
    t = np.linspace(0.0, 1.0, nquad)
    P = np.empty(wl.N)
    for k0 in range(0, wl.N, 2048):
        xs, ys = x[k0:k0 + 2048, None], y[k0:k0 + 2048, None]
        yy = ys + (2.0 - ys) * t[None, :]
        rho = rho2 + (rho1 - rho2) * tanh_profile(np.hypot(xs, yy - 0.5) - R, wl.eps)
        P[k0:k0 + 2048] = P_top + g * _trapezoid(rho, yy)
    wl.w = conserved(wl, phi, s, P, 0.0, 0.0)
    wl.dt = stable_dt(wl, 0.0, P_top)
    wl.meta = dict(P_top=P_top, case=case)
    return wl


def resized(wl_fn, **kw) -> Workload:
    """Convenience: build a workload with overridden sizes (used for small parity cases)."""
    return wl_fn(**kw)


def ensemble(n: int = 256, seed: int = 4, nmin: int = 16, nmax: int = 128, orders=(2, 3, 4, 5),
             Rmin: float = 0.05, Rmax: float = 0.2, u: float = 1.0, v: float = 0.5, P0: float = 1e5,
             nsteps: int = 200) -> list:
    """Independent 2D periodic drop / bubble problems with seeded sizes, orders, radii and centres:
    N ~ U{nmin..nmax} (N x N quads), p ~ U(orders), water drop in air or air bubble in water
    (half each), R ~ U[Rmin, Rmax], centre ~ U[0, 1]^2, eps = 0.75 h, own dt per problem."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        N = int(rng.integers(nmin, nmax + 1))
        p = int(rng.choice(orders))
        bubble = bool(rng.integers(0, 2))
        R = float(rng.uniform(Rmin, Rmax))
        c = rng.uniform(0.0, 1.0, size=2)
        wl = drop_2d(n=N, p=p, R=R, u=u, v=v, P0=P0, nsteps=nsteps, center=c, water_inside=not bubble)
        wl.name = f"ens{k}_{N}x{N}p{p}{'b' if bubble else 'd'}"
        wl.meta.update(kind="bubble" if bubble else "drop", member=k, seed=seed)
        out.append(wl)
    return out


def level_set_modes(wl: Workload, cx: float, cy: float):
    """cos(k theta), sin(k theta), k = 1..8, of the polar angle about (cx, cy) (periodic
    minimum image) at every node: shape (16, N), rows ordered (cos 1, sin 1, cos 2, ...)."""
    x, y = node_coords(wl)
    dx = x - cx
    dy = y - cy
    dx -= np.round(dx)
    dy -= np.round(dy)
    th = np.arctan2(dy, dx)
    rows = []
    for k in range(1, 9):
        rows += [np.cos(k * th), np.sin(k * th)]
    return np.array(rows)


def adjoint_drop(n: int = 128, p: int = 3, seed: int = 5, theta=None, nsteps: int = 200, R: float = 0.15,
                 u: float = 1.0, v: float = 0.5, P0: float = 1e5, eps_h: float = 0.75) -> Workload:
    """Drop advection with a parametrised initial level set: psi0 = r - R - sum_k (theta_{2k-1} cos k th +
    theta_{2k} sin k th) about the (seeded) drop centre, phi0 the tanh profile of r - R.
    theta defaults to 16 draws of N(0, 0.01^2) from seed 50."""
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0.0, 1.0, size=2)
    if theta is None:
        theta = np.random.default_rng(50).normal(0.0, 0.01, size=16)
    wl = drop_2d(n=n, p=p, R=R, u=u, v=v, P0=P0, eps_h=eps_h, nsteps=nsteps, center=(cx, cy))
    x, y = node_coords(wl)
    modes = level_set_modes(wl, cx, cy)
    w = wl.w.copy()
    w[1] = w[1] - np.asarray(theta) @ modes
    wl.w = w
    wl.meta.update(theta=list(map(float, theta)), seed=seed)
    return wl


# ---------------------------------------------------------------------------
# Kinematic mode (Sec. 4.1): phase field and level set, prescribed velocity
# ---------------------------------------------------------------------------

@dataclass
class KinWorkload:
    """A kinematic-mode problem: periodic 2D mesh, order, Allen-Cahn constants, prescribed
    velocity (kind "uniform" with (u0, v0), or "rider_kothe" with period T), the initial
    (phi, psi) state (2, N) and a time step."""
    name: str
    nx: int
    ny: int
    p: int
    x0: float = -0.5
    x1: float = 0.5
    y0: float = -0.5
    y1: float = 0.5
    Gamma: float = 1.0
    eps: float = 0.05
    c_ip: float = 1.0
    vel: str = "rider_kothe"
    u0: float = 0.0
    v0: float = 0.0
    T: float = 4.0
    xc: float = 0.0           # Rider-Kothe vortex centre
    yc: float = 0.0
    w: Optional[np.ndarray] = None
    dt: float = 0.0
    nsteps: int = 0
    meta: dict = field(default_factory=dict)
    dim: int = 2
    elem: str = "quad"        # "quad": the rectangles (mesh (a)); "tri": each split in two (mesh (b))

    @property
    def Np(self) -> int:
        return (self.p + 1) * (self.p + 2) // 2 if self.elem == "tri" else (self.p + 1) ** 2

    @property
    def E(self) -> int:
        return self.nx * self.ny * (2 if self.elem == "tri" else 1)

    @property
    def N(self) -> int:
        return self.E * self.Np

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def problem_kwargs(self) -> dict:
        """The oracle's problem description (periodic 2D mesh and the Allen-Cahn constants)."""
        return dict(dim=2, nx=self.nx, ny=self.ny, p=self.p, x0=self.x0, x1=self.x1, y0=self.y0, y1=self.y1,
                    Gamma=self.Gamma, eps=self.eps, c_ip=self.c_ip)

    def velocity_kwargs(self) -> dict:
        return dict(kind=self.vel, u0=self.u0, v0=self.v0, T=self.T, xc=self.xc, yc=self.yc)


def kin_stable_dt(wl: KinWorkload, umax: float) -> float:
    """Advective limit 0.5 h / ((2p + 1) |u|max) and the parabolic limit of the SIP term (h the
    cell width); on triangles 0.4 of that (the split cells run stably up to about 0.7 of it for
    p <= 3 and 0.5 for p = 4 on the Rider-Kothe drop)."""
    h = min(wl.hx, wl.hy)
    q = 2 * wl.p + 1
    dt = 0.5 * h / (q * max(umax, 1e-12))
    if wl.Gamma * wl.eps > 0:
        dt = min(dt, 0.1 * h * h / (q * q * wl.Gamma * wl.eps))
    return dt * (0.4 if wl.elem == "tri" else 1.0)


def rider_kothe(n: int = 16, p: int = 3, T: float = 4.0, R: float = 0.15, center=(0.0, 0.25),
                eps_dof: float = 0.75, Gamma: float = 1.0, vortex=(0.0, 0.0), elem: str = "quad",
                eps_h: Optional[float] = None) -> KinWorkload:
    """Rider-Kothe vortex (Sec. 4.1): a drop of radius 0.15 centred at (0, 0.25) in the periodic
    square [-0.5, 0.5]^2, stretched by the time-reversing vortex of period T = 4 centred at
    `vortex` (the domain centre; (0.5, 0.5) gives the printed formula, whose vortex sits at the
    domain corners).  Phase 1 is the drop; psi = R - r grows into it.  The paper leaves eps and
    Gamma unstated for this test: eps = eps_dof h / (p + 1), 0.75 of the node spacing h / (p + 1)
    (h: cell width; the paper compares orders at matched degrees of freedom), or eps_h h when
    eps_h is given; Gamma = |u|max = 1."""
    wl = KinWorkload(name=f"rk2d_{n}x{n}p{p}" + ("tri" if elem == "tri" else ""), nx=n, ny=n, p=p, Gamma=Gamma,
                     vel="rider_kothe", T=T, xc=vortex[0], yc=vortex[1], elem=elem)
    wl.eps = eps_h * wl.hx if eps_h is not None else eps_dof * wl.hx / (p + 1)
    x, y = _kin_nodes(wl)
    r = np.hypot(x - center[0], y - center[1])
    s = R - r
    wl.w = np.stack([tanh_profile(s, wl.eps), s])
    wl.dt = kin_stable_dt(wl, 1.0)
    wl.nsteps = int(np.ceil(T / wl.dt))
    wl.dt = T / wl.nsteps
    wl.meta = dict(R=R, center=center)
    return wl


def kin_drop(n: int = 16, p: int = 3, R: float = 0.15, u0: float = 1.0, v0: float = 0.0,
             eps: float = 0.05, Gamma: float = 1.0) -> KinWorkload:
    """Linear advection of a droplet (Sec. 4.1): radius 0.15 at the origin of the periodic square
    [-0.5, 0.5]^2, constant velocity (1, 0), eps = 0.05; one period is t = 1."""
    wl = KinWorkload(name=f"kdrop2d_{n}x{n}p{p}", nx=n, ny=n, p=p, Gamma=Gamma, eps=eps, vel="uniform",
                     u0=u0, v0=v0)
    x, y = _kin_nodes(wl)
    s = R - np.hypot(x, y)
    wl.w = np.stack([tanh_profile(s, eps), s])
    wl.dt = kin_stable_dt(wl, np.hypot(u0, v0))
    wl.nsteps = int(np.ceil(1.0 / wl.dt))
    wl.dt = 1.0 / wl.nsteps
    return wl


def _kin_nodes(wl: KinWorkload):
    if wl.elem == "tri":
        return _tri_nodes(wl)
    xi = gll_points(wl.p)
    P1 = wl.p + 1
    e = np.arange(wl.nx * wl.ny)
    ex, ey = e % wl.nx, e // wl.nx
    a = np.arange(P1 * P1)
    i, j = a % P1, a // P1
    x = wl.x0 + wl.hx * (ex[:, None] + 0.5 * (xi[i][None, :] + 1.0))
    y = wl.y0 + wl.hy * (ey[:, None] + 0.5 * (xi[j][None, :] + 1.0))
    return x.ravel(), y.ravel()


def _tri_nodes(wl: KinWorkload):
    """Equispaced nodes of the split-rectangle triangles: cell (i, j) gives triangle 2 (i + nx j)
    with vertices (x_i, y_j), (x_i+1, y_j), (x_i+1, y_j+1) and triangle 2 (i + nx j) + 1 with
    (x_i, y_j), (x_i+1, y_j+1), (x_i, y_j+1); node (a, b), a + b <= p, a fastest, at barycentric
    weights (1 - (a + b)/p, a/p, b/p) of the three vertices."""
    p = wl.p
    a = np.array([i for j in range(p + 1) for i in range(p + 1 - j)], dtype=float) / p
    b = np.array([j for j in range(p + 1) for i in range(p + 1 - j)], dtype=float) / p
    cell = np.arange(wl.nx * wl.ny)
    xa = wl.x0 + (cell % wl.nx) * wl.hx
    ya = wl.y0 + (cell // wl.nx) * wl.hy
    x = np.empty((wl.nx * wl.ny, 2, len(a)))
    y = np.empty_like(x)
    x[:, 0] = xa[:, None] + wl.hx * (a + b)[None, :]
    y[:, 0] = ya[:, None] + wl.hy * b[None, :]
    x[:, 1] = xa[:, None] + wl.hx * a[None, :]
    y[:, 1] = ya[:, None] + wl.hy * (a + b)[None, :]
    return x.ravel(), y.ravel()

