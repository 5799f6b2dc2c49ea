"""FP64 CPU oracle for the DG right-hand side (Tonicello & Ihme, arXiv 2306.05002).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users of this package; the product
path (``paper_2306_05002_gb300``) never imports it, and this package imports
nothing from the product.  The arithmetic lives in ``dg_oracle.c`` (plain C,
FP64, compiled with FMA contraction disabled); this module only marshals numpy
arrays through ctypes.

Parity status of each function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants of the paper's scheme (Sec. 3: interface equilibrium,
conservation, free stream), the symmetry of the SIP bilinear form, textbook
limits of the stiffened-gas closure and convergence rates.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_SRC_TRI = os.path.join(_HERE, "dg_oracle_tri.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

BC = {"periodic": 0, "noslip": 1, "slip": 2, "pressure": 3}
NV = 7


CFLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared"]


def compile_sources(sources, out: str, openmp: bool = False, include_dir: str | None = None) -> str:
    """Compile C sources of the oracle into the shared library `out` (gcc, FP64, no FMA
    contraction: every product and sum is rounded on its own, as written)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc"] + CFLAGS + (["-fopenmp"] if openmp else []) + (["-I" + include_dir] if include_dir else [])
    subprocess.check_call(cmd + ["-o", tmp] + list(sources) + ["-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so``, or, with ``openmp``, the same source
    with its element loops parallel into ``oracle/liboracle_omp.so`` (used only to time the
    oracle on all host cores; the tests pin the plain build)."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC_TRI), os.path.getmtime(os.path.join(_HERE, "dg_oracle.h"))
    ):
        compile_sources([_SRC, _SRC_TRI], out, openmp=openmp)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("p", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("gamma", ctypes.c_double * 2), ("pinf", ctypes.c_double * 2),
        ("rho0", ctypes.c_double * 2), ("mu", ctypes.c_double * 2),
        ("sigma", ctypes.c_double), ("g", ctypes.c_double * 2),
        ("Gamma", ctypes.c_double), ("eps", ctypes.c_double), ("c_ip", ctypes.c_double),
        ("viscous", ctypes.c_int), ("gravity", ctypes.c_int), ("surface_tension", ctypes.c_int),
        ("p_bc", ctypes.c_double * 4), ("grad_lift", ctypes.c_int),
    ]


@dataclass
class Problem:
    """Plain description of one DG problem (mesh, order, closure, model constants)."""
    dim: int = 2
    nx: int = 4
    ny: int = 4
    p: int = 3
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
    p_bc: tuple = (0.0, 0.0, 0.0, 0.0)
    grad_lift: bool = False

    @property
    def Np(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.Np

    def _c(self) -> _Problem:
        s = _Problem()
        s.dim, s.nx, s.ny, s.p = self.dim, self.nx, self.ny, self.p
        s.x0, s.x1, s.y0, s.y1 = self.x0, self.x1, self.y0, self.y1
        for i, b in enumerate(self.bc):
            s.bc[i] = BC[b] if isinstance(b, str) else int(b)
        for i in range(2):
            s.gamma[i], s.pinf[i] = self.gamma[i], self.pinf[i]
            s.rho0[i], s.mu[i], s.g[i] = self.rho0[i], self.mu[i], self.g[i]
        s.sigma, s.Gamma, s.eps, s.c_ip = self.sigma, self.Gamma, self.eps, self.c_ip
        s.viscous, s.gravity, s.surface_tension = int(self.viscous), int(self.gravity), int(self.surface_tension)
        for i in range(4):
            s.p_bc[i] = self.p_bc[i]
        s.grad_lift = int(self.grad_lift)
        return s


class _Velocity(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u0", ctypes.c_double), ("v0", ctypes.c_double), ("T", ctypes.c_double),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double)]


VEL = {"uniform": 0, "rider_kothe": 1}


@dataclass
class Velocity:
    """Prescribed velocity of the kinematic mode (Sec. 4.1): uniform (u0, v0), or the
    Rider-Kothe vortex with period T about the centre (xc, yc) (0.5, 0.5: the printed formula)."""
    kind: str = "uniform"
    u0: float = 1.0
    v0: float = 0.0
    T: float = 4.0
    xc: float = 0.5
    yc: float = 0.5

    def _c(self) -> _Velocity:
        s = _Velocity()
        s.kind, s.u0, s.v0, s.T, s.xc, s.yc = VEL[self.kind], self.u0, self.v0, self.T, self.xc, self.yc
        return s


_libs = {}


def _configure(_lib):
    """Declare the argument types of every exported oracle function on a loaded library."""
    _lib.orc_threads.argtypes = [ctypes.c_int]
    _lib.orc_threads.restype = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(_Problem)
    _lib.orc_gll.argtypes = [ctypes.c_int, dp, dp]
    _lib.orc_lagrange_deriv.argtypes = [ctypes.c_int, dp, dp]
    _lib.orc_num_nodes.argtypes = [pp]
    _lib.orc_num_nodes.restype = ctypes.c_long
    _lib.orc_nodes.argtypes = [pp, dp, dp]
    _lib.orc_primitives.argtypes = [pp, dp, dp]
    _lib.orc_gradients.argtypes = [pp, dp, dp, dp]
    _lib.orc_rhs.argtypes = [pp, dp, dp, dp, dp]
    _lib.orc_rk3.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int]
    _lib.orc_diag.argtypes = [pp, dp, dp]
    vp = ctypes.POINTER(_Velocity)
    _lib.orc_velocity_at.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
    _lib.orc_velocity_at.restype = None
    _lib.orc_stream_at.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    _lib.orc_stream_at.restype = ctypes.c_double
    _lib.orc_kin_velocity.argtypes = [pp, vp, ctypes.c_double, dp, dp]
    _lib.orc_kin_rhs.argtypes = [pp, vp, ctypes.c_double, dp, dp, dp]
    _lib.orc_kin_rk4.argtypes = [pp, vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    _lib.orc_tri_num_nodes.argtypes = [pp]
    _lib.orc_tri_num_nodes.restype = ctypes.c_long
    _lib.orc_tri_nodes.argtypes = [pp, dp, dp]
    _lib.orc_tri_integral.argtypes = [pp, dp, dp]
    _lib.orc_tri_mass.argtypes = [pp, ctypes.c_int, dp]
    _lib.orc_tri_rhs.argtypes = [pp, vp, ctypes.c_double, dp, dp, dp]
    _lib.orc_tri_rk4.argtypes = [pp, vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    _lib.orc_reinit_sign.argtypes = [pp, dp, dp]
    _lib.orc_reinit_rhs.argtypes = [pp, dp, dp, ctypes.c_double, dp]
    _lib.orc_reinit.argtypes = [pp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    return _lib


def lib(openmp: bool = False):
    """The plain oracle library, or (``openmp``) its OpenMP build."""
    _lib = _libs.get(openmp)
    if _lib is None:
        _lib = _libs[openmp] = _configure(ctypes.CDLL(build(openmp=openmp)))
    return _lib


@contextlib.contextmanager
def using(path: str):
    """Route every function of this module through the library at `path` (another build of
    the oracle sources) for the duration of the block.  The mutation tests use it to run the
    pins against copies of the oracle with a planted mistake."""
    saved = _libs.get(False)
    _libs[False] = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        if saved is None:
            _libs.pop(False, None)
        else:
            _libs[False] = saved


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def gll(p: int):
    """GLL nodes and weights on [-1, 1]."""
    xi = np.zeros(p + 1)
    wt = np.zeros(p + 1)
    _check(lib().orc_gll(p, _ptr(xi), _ptr(wt)), "gll")
    return xi, wt


def lagrange_deriv(p: int, xi):
    """D[a, b] = l_b'(xi_a)."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    D = np.zeros((p + 1, p + 1))
    _check(lib().orc_lagrange_deriv(p, _ptr(xi), _ptr(D)), "lagrange_deriv")
    return D


def nodes(pb: Problem):
    x = np.zeros(pb.N)
    y = np.zeros(pb.N)
    s = pb._c()
    _check(lib().orc_nodes(ctypes.byref(s), _ptr(x), _ptr(y)), "nodes")
    return x, y


def primitives(pb: Problem, w):
    """rho, u, v, P, c, B at every node, shape (6, N)."""
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(NV, pb.N)
    out = np.zeros((6, pb.N))
    s = pb._c()
    _check(lib().orc_primitives(ctypes.byref(s), _ptr(w), _ptr(out)), "primitives")
    return out


def gradients(pb: Problem, f):
    """Gradient (gx, gy) of the nodal field f: broken, or BR1-lifted when pb.grad_lift."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(pb.N)
    gx, gy = np.zeros(pb.N), np.zeros(pb.N)
    s = pb._c()
    _check(lib().orc_gradients(ctypes.byref(s), _ptr(f), _ptr(gx), _ptr(gy)), "gradients")
    return gx, gy


def rhs(pb: Problem, w, want_scale: bool = False, want_parts: bool = False):
    """L = M^-1 R(w), shape (7, N); optionally the rounding scale S and the parts."""
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(NV, pb.N)
    L = np.zeros((NV, pb.N))
    S = np.zeros((NV, pb.N)) if want_scale else None
    parts = np.zeros((3, NV, pb.N)) if want_parts else None
    s = pb._c()
    _check(lib().orc_rhs(ctypes.byref(s), _ptr(w), _ptr(L), _ptr(S), _ptr(parts)), "rhs")
    out = [L]
    if want_scale:
        out.append(S)
    if want_parts:
        out.append(parts)
    return out[0] if len(out) == 1 else tuple(out)


def rk3(pb: Problem, w, dt: float, nsteps: int, threads: int = 0):
    """Return w after nsteps SSP-RK3 steps (input left untouched).  threads > 0 runs the OpenMP
    build on that many threads (bit-identical results)."""
    w = np.array(w, dtype=np.float64).reshape(NV, pb.N).copy()
    s = pb._c()
    L = lib(openmp=threads > 0)
    if threads > 0:
        L.orc_threads(int(threads))
    _check(L.orc_rk3(ctypes.byref(s), _ptr(w), float(dt), int(nsteps)), "rk3")
    return w


def rhs_threads(pb: Problem, w, threads: int):
    """The right-hand side from the OpenMP build on `threads` threads (for its bitwise check)."""
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(NV, pb.N)
    L = np.zeros((NV, pb.N))
    s = pb._c()
    lb = lib(openmp=True)
    lb.orc_threads(int(threads))
    _check(lb.orc_rhs(ctypes.byref(s), _ptr(w), _ptr(L), None, None), "rhs")
    return L


def diag(pb: Problem, w):
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(NV, pb.N)
    out = np.zeros(16)
    s = pb._c()
    _check(lib().orc_diag(ctypes.byref(s), _ptr(w), _ptr(out)), "diag")
    return out


def velocity_at(vel: Velocity, x: float, y: float, t: float):
    u, v = ctypes.c_double(), ctypes.c_double()
    c = vel._c()
    lib().orc_velocity_at(ctypes.byref(c), float(x), float(y), float(t), ctypes.byref(u), ctypes.byref(v))
    return u.value, v.value


def stream_at(vel: Velocity, x: float, y: float, t: float) -> float:
    """Stream function of the prescribed velocity: u = dPsi/dy, v = -dPsi/dx."""
    c = vel._c()
    return lib().orc_stream_at(ctypes.byref(c), float(x), float(y), float(t))


def kin_velocity(pb: Problem, vel: Velocity, t: float):
    """The nodal velocity (u, v) the kinematic scheme uses at time t, shape (2, N)."""
    out = np.zeros((2, pb.N))
    s, c = pb._c(), vel._c()
    _check(lib().orc_kin_velocity(ctypes.byref(s), ctypes.byref(c), float(t), _ptr(out[0]), _ptr(out[1])),
           "kin_velocity")
    return out


def kin_rhs(pb: Problem, vel: Velocity, t: float, w, want_scale: bool = False):
    """Kinematic mode: L = M^-1 R(w) at time t for w = (phi, psi), shape (2, N)."""
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(2, pb.N)
    L = np.zeros((2, pb.N))
    S = np.zeros((2, pb.N)) if want_scale else None
    s, c = pb._c(), vel._c()
    _check(lib().orc_kin_rhs(ctypes.byref(s), ctypes.byref(c), float(t), _ptr(w), _ptr(L), _ptr(S)), "kin_rhs")
    return (L, S) if want_scale else L


def kin_rk4(pb: Problem, vel: Velocity, w, t0: float, dt: float, nsteps: int):
    """Return (phi, psi) after nsteps classical RK4 steps from time t0 (input left untouched)."""
    w = np.array(w, dtype=np.float64).reshape(2, pb.N).copy()
    s, c = pb._c(), vel._c()
    _check(lib().orc_kin_rk4(ctypes.byref(s), ctypes.byref(c), _ptr(w), float(t0), float(dt), int(nsteps)),
           "kin_rk4")
    return w


def reinit_sign(pb: Problem, phi):
    """Smeared sign S = tanh(psi0 / (2 eps |grad psi0|)) of psi0 = phi - 1/2 at every node."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(pb.N)
    S = np.zeros(pb.N)
    s = pb._c()
    _check(lib().orc_reinit_sign(ctypes.byref(s), _ptr(phi), _ptr(S)), "reinit_sign")
    return S


def reinit_rhs(pb: Problem, S, psi, nu: float):
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(pb.N)
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(pb.N)
    L = np.zeros(pb.N)
    s = pb._c()
    _check(lib().orc_reinit_rhs(ctypes.byref(s), _ptr(S), _ptr(psi), float(nu), _ptr(L)), "reinit_rhs")
    return L


def reinit(pb: Problem, phi, niter: int, nu: float, dtau: float):
    """psi after niter pseudo-time SSP-RK3 steps from psi0 = phi - 1/2."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(pb.N)
    psi = np.zeros(pb.N)
    s = pb._c()
    _check(lib().orc_reinit(ctypes.byref(s), _ptr(phi), _ptr(psi), int(niter), float(nu), float(dtau)), "reinit")
    return psi


def tri_num_nodes(pb: Problem) -> int:
    return int(lib().orc_tri_num_nodes(ctypes.byref(pb._c())))


def tri_nodes(pb: Problem):
    """Node coordinates of the triangulated mesh (kinematic mode on triangles)."""
    N = tri_num_nodes(pb)
    x, y = np.zeros(N), np.zeros(N)
    s = pb._c()
    _check(lib().orc_tri_nodes(ctypes.byref(s), _ptr(x), _ptr(y)), "tri_nodes")
    return x, y


def tri_integral(pb: Problem, f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = ctypes.c_double()
    s = pb._c()
    _check(lib().orc_tri_integral(ctypes.byref(s), _ptr(f), ctypes.byref(out)), "tri_integral")
    return out.value


def tri_mass(pb: Problem, e: int):
    """Mass matrix int l_i l_j of triangle e."""
    Np = (pb.p + 1) * (pb.p + 2) // 2
    M = np.zeros((Np, Np))
    s = pb._c()
    _check(lib().orc_tri_mass(ctypes.byref(s), int(e), _ptr(M)), "tri_mass")
    return M


def tri_rhs(pb: Problem, vel: Velocity, t: float, w, want_scale: bool = False):
    N = tri_num_nodes(pb)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(2, N)
    L = np.zeros((2, N))
    S = np.zeros((2, N)) if want_scale else None
    s, c = pb._c(), vel._c()
    _check(lib().orc_tri_rhs(ctypes.byref(s), ctypes.byref(c), float(t), _ptr(w), _ptr(L), _ptr(S)), "tri_rhs")
    return (L, S) if want_scale else L


def tri_rk4(pb: Problem, vel: Velocity, w, t0: float, dt: float, nsteps: int):
    N = tri_num_nodes(pb)
    w = np.array(w, dtype=np.float64).reshape(2, N).copy()
    s, c = pb._c(), vel._c()
    _check(lib().orc_tri_rk4(ctypes.byref(s), ctypes.byref(c), _ptr(w), float(t0), float(dt), int(nsteps)),
           "tri_rk4")
    return w

