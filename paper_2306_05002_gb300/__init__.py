"""GB300-native DG solver for diffused-interface two-phase flow.

Tonicello & Ihme, "A high-order diffused-interface approach for two-phase
compressible flow simulations using a Discontinuous Galerkin framework"
(arXiv 2306.05002): the explicit DG right-hand side of the quasi-conservative
five-equation model with the Allen-Cahn phase field and an advected level set,
and its SSP-RK3 step, as hand-written sm_103a CUDA kernels behind the C ABI of
``include/dgpf.h`` (``libdgpf.so``).

This module is a thin ctypes binding with the C names (``dg_create``,
``dg_rhs``, ``dg_step``, ...): it marshals arguments only.  Every step of the
right-hand side runs in the library's kernels; there is no CPU fallback, and
using the binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

from . import workloads  # noqa: F401  (numpy-only input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgpf.so")
# The bounds-checked build (same sources with -DDG_CHECK), loaded instead of LIB_PATH when the
# environment sets DGPF_CHECKED=1.
LIB_CHECK_PATH = os.path.join(_HERE, "libdgpf_check.so")

DG_OK = 0
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_CUDA", -3: "DG_ERR_OOM", -4: "DG_ERR_TIMEOUT",
          -5: "DG_ERR_NONFINITE", -6: "DG_ERR_NONPHYSICAL", -7: "DG_ERR_UNSUPPORTED", -8: "DG_ERR_BOUNDS"}
BC = {"periodic": 0, "noslip": 1, "slip": 2, "pressure": 3}
PREC = {"fp64": 0, "fp32bulk": 1}

# Every exported symbol of include/dgpf.h.
EXPORTS = ["dg_create", "dg_destroy", "dg_state_len", "dg_rhs", "dg_step", "dg_step_host", "dg_diag",
           "dg_status_read", "dg_last_error", "dg_time_kernels", "dg_kernel_costs", "dg_step_launches",
           "dg_rhs_noalloc", "dg_batch_create",
           "dg_batch_step", "dg_rhs_vjp", "dg_adjoint_step", "dg_tape_len", "dg_step_tape",
           "dg_adjoint_step_tape", "dg_adjoint_segment", "dg_batch_tiles", "dg_kin_create", "dg_kin_rhs",
           "dg_kin_step", "dg_kin_nodes", "dg_reinit", "dg_peak_flops", "dg_check_build",
           "dg_check_selftest"]


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dg_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("p_bc", ctypes.c_double * 4), ("elem", ctypes.c_int)]


class dg_eos(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double * 2), ("pinf", ctypes.c_double * 2), ("rho0", ctypes.c_double * 2),
                ("mu", ctypes.c_double * 2), ("sigma", ctypes.c_double), ("g", ctypes.c_double * 2)]


class dg_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("c_ip", ctypes.c_double), ("viscous", ctypes.c_int),
                ("gravity", ctypes.c_int), ("surface_tension", ctypes.c_int), ("check_finite", ctypes.c_int),
                ("batch_tile", ctypes.c_int), ("grad_lift", ctypes.c_int)]


class dg_velocity(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u0", ctypes.c_double), ("v0", ctypes.c_double), ("T", ctypes.c_double),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double)]


VEL = {"uniform": 0, "rider_kothe": 1}

_lib = None


def load(path: str | None = None):
    """Load libdgpf.so (built by ``paper_2306_05002_gb300.build``), or libdgpf_check.so when the
    environment sets DGPF_CHECKED=1; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or (LIB_CHECK_PATH if os.environ.get("DGPF_CHECKED") == "1" else LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t
    lib.dg_create.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int, ctypes.POINTER(dg_eos), ctypes.c_double,
                              ctypes.c_double, ctypes.POINTER(dg_opts), ctypes.POINTER(vp)]
    lib.dg_create.restype = ctypes.c_int
    lib.dg_destroy.argtypes = [vp]
    lib.dg_destroy.restype = None
    lib.dg_state_len.argtypes = [vp]
    lib.dg_state_len.restype = sz
    lib.dg_rhs.argtypes = [vp, dp, dp, vp]
    lib.dg_rhs.restype = ctypes.c_int
    lib.dg_step.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int, vp]
    lib.dg_step.restype = ctypes.c_int
    lib.dg_step_host.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int, vp]
    lib.dg_step_host.restype = ctypes.c_int
    lib.dg_diag.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_double), vp]
    lib.dg_diag.restype = ctypes.c_int
    lib.dg_status_read.argtypes = [vp, vp]
    lib.dg_status_read.restype = ctypes.c_int
    lib.dg_last_error.argtypes = [vp]
    lib.dg_last_error.restype = ctypes.c_char_p
    lib.dg_time_kernels.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, vp]
    lib.dg_time_kernels.restype = ctypes.c_int
    lib.dg_kernel_costs.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_int]
    lib.dg_kernel_costs.restype = ctypes.c_int
    lib.dg_step_launches.argtypes = [vp, ctypes.c_int]
    lib.dg_step_launches.restype = ctypes.c_int
    lib.dg_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(dg_mesh), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(dg_eos), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(dg_opts), ctypes.POINTER(vp)]
    lib.dg_batch_create.restype = ctypes.c_int
    lib.dg_batch_step.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_int, vp]
    lib.dg_batch_step.restype = ctypes.c_int
    ip, dpp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.dg_kin_create.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(dg_velocity), ctypes.c_double, ctypes.POINTER(vp)]
    lib.dg_kin_create.restype = ctypes.c_int
    lib.dg_kin_nodes.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int, dp, dp]
    lib.dg_kin_nodes.restype = ctypes.c_int
    lib.dg_kin_rhs.argtypes = [vp, dp, ctypes.c_double, dp, vp]
    lib.dg_kin_rhs.restype = ctypes.c_int
    lib.dg_kin_step.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    lib.dg_kin_step.restype = ctypes.c_int
    lib.dg_reinit.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
    lib.dg_reinit.restype = ctypes.c_int
    lib.dg_batch_tiles.argtypes = [vp, ip, ip, ip, dpp, dpp, ctypes.c_int]
    lib.dg_batch_tiles.restype = ctypes.c_int
    lib.dg_rhs_vjp.argtypes = [vp, dp, dp, dp, vp]
    lib.dg_rhs_vjp.restype = ctypes.c_int
    lib.dg_adjoint_step.argtypes = [vp, dp, dp, dp, ctypes.c_double, vp]
    lib.dg_adjoint_step.restype = ctypes.c_int
    lib.dg_tape_len.argtypes = [vp]
    lib.dg_tape_len.restype = sz
    lib.dg_step_tape.argtypes = [vp, dp, ctypes.c_double, dp, vp]
    lib.dg_step_tape.restype = ctypes.c_int
    lib.dg_adjoint_step_tape.argtypes = [vp, dp, dp, dp, dp, ctypes.c_double, vp]
    lib.dg_adjoint_step_tape.restype = ctypes.c_int
    lib.dg_adjoint_segment.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, dp, dp, dp, vp]
    lib.dg_adjoint_segment.restype = ctypes.c_int
    lib.dg_peak_flops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    lib.dg_peak_flops.restype = ctypes.c_int
    lib.dg_check_build.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    lib.dg_check_build.restype = ctypes.c_int
    lib.dg_check_selftest.argtypes = [vp]
    lib.dg_check_selftest.restype = ctypes.c_int
    _lib = lib
    return lib


def check_build():
    """(is_checked_build, bounds failures reported so far in this process): dg_check_build."""
    n = ctypes.c_longlong()
    flag = load().dg_check_build(ctypes.byref(n))
    return bool(flag), n.value


def peak_flops(kind: str = "fp64", iters: int = 0, stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (dg_peak_flops): kind "fp64" or "fp32"."""
    k = {"fp64": 0, "fp32": 1}[kind]
    out = ctypes.c_double()
    n = iters or (20000 if k == 0 else 400000)
    _check(None, load().dg_peak_flops(k, n, ctypes.byref(out), _stream(stream)), "dg_peak_flops")
    return out.value


def _check(ctx, status, what):
    if status != DG_OK:
        msg = load().dg_last_error(ctx)
        raise DGError(status, f"{what}: {msg.decode() if msg else ''}")


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


_raw_stream = None


def _stream(stream=None):
    """The CUDA stream handle of `stream`, or of torch's current stream on the current device.  The
    current stream's handle is read with torch's raw-handle query where it exists: building a
    torch Stream object per call costs microseconds of host time on every library call."""
    global _raw_stream
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    import torch
    if _raw_stream is None:
        _raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", False)
    if _raw_stream:
        return ctypes.c_void_p(_raw_stream(torch.cuda.current_device()))
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_structs(dim, nx, ny, x0, x1, y0, y1, bc, gamma, pinf, rho0, mu=(0.0, 0.0), sigma=0.0, g=(0.0, 0.0),
                 precision="fp64", c_ip=1.0, viscous=False, gravity=False, surface_tension=False,
                 check_finite=True, p_bc=(0.0, 0.0, 0.0, 0.0), grad_lift=False, **_ignored):
    m = dg_mesh()
    m.dim, m.nx, m.ny = dim, nx, ny
    m.x0, m.x1, m.y0, m.y1 = x0, x1, y0, y1
    for i, b in enumerate(bc):
        m.bc[i] = BC[b] if isinstance(b, str) else int(b)
        m.p_bc[i] = float(p_bc[i])
    e = dg_eos()
    for i in range(2):
        e.gamma[i], e.pinf[i], e.rho0[i], e.mu[i], e.g[i] = gamma[i], pinf[i], rho0[i], mu[i], g[i]
    e.sigma = sigma
    o = dg_opts()
    o.prec = PREC[precision] if isinstance(precision, str) else int(precision)
    o.c_ip, o.viscous, o.gravity, o.surface_tension = c_ip, int(viscous), int(gravity), int(surface_tension)
    o.check_finite = int(check_finite)
    o.grad_lift = int(grad_lift)
    return m, e, o


class Solver:
    """One DG problem on the current CUDA device (wraps a ``dg_ctx``).

    ``problem`` is a :class:`workloads.Workload` (or any object with the same
    fields).  State tensors are float64 CUDA tensors of shape (7, N).
    """

    def __init__(self, problem, precision: str = "fp64", check_finite: bool = True):
        lib = load()
        kw = problem.problem_kwargs() if hasattr(problem, "problem_kwargs") else dict(problem)
        p = kw.pop("p")
        Gamma, eps = kw.pop("Gamma"), kw.pop("eps")
        m, e, o = make_structs(precision=precision, check_finite=check_finite, **kw)
        self._m, self._e, self._o = m, e, o
        h = ctypes.c_void_p()
        st = lib.dg_create(ctypes.byref(m), p, ctypes.byref(e), Gamma, eps, ctypes.byref(o), ctypes.byref(h))
        _check(None, st, "dg_create")
        self.ctx = h
        self.len = lib.dg_state_len(h)
        self.N = self.len // 7

    def close(self):
        self._adjoint_workspace = None
        if getattr(self, "ctx", None):
            load().dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dg_rhs(self, w, L=None, stream=None):
        import torch
        if L is None:
            L = torch.empty_like(w)
        _check(self.ctx, load().dg_rhs(self.ctx, _ptr(w), _ptr(L), _stream(stream)), "dg_rhs")
        return L

    def dg_step(self, w, dt: float, nsteps: int, stream=None):
        """Advance w in place.  A CPU tensor goes through dg_step_host: a pinned one is read and
        written in place by the FP32-bulk kernels, otherwise it is staged through the device."""
        import torch
        if w.is_cuda:
            _check(self.ctx, load().dg_step(self.ctx, _ptr(w), float(dt), int(nsteps), _stream(stream)), "dg_step")
            return w
        if w.dtype != torch.float64 or not w.is_contiguous() or w.numel() != self.len:
            raise ValueError("dg_step: host state must be a contiguous float64 tensor of dg_state_len values")
        _check(self.ctx, load().dg_step_host(self.ctx, ctypes.c_void_p(w.data_ptr()), float(dt), int(nsteps),
                                             _stream(stream)), "dg_step_host")
        return w

    def dg_rhs_vjp(self, w, lam, out=None, stream=None):
        """out = (dL/dw)^T lam (FP64 contexts without viscous / surface-tension terms)."""
        import torch
        if out is None:
            out = torch.empty_like(w)
        _check(self.ctx, load().dg_rhs_vjp(self.ctx, _ptr(w), _ptr(lam), _ptr(out), _stream(stream)), "dg_rhs_vjp")
        return out

    def dg_adjoint_step(self, w_n, lam_np1, dt: float, lam_n=None, stream=None):
        """lam_n = (d w_{n+1} / d w_n)^T lam_np1 for one SSP-RK3 step of size dt from w_n."""
        import torch
        if lam_n is None:
            lam_n = torch.empty_like(w_n)
        _check(self.ctx, load().dg_adjoint_step(self.ctx, _ptr(w_n), _ptr(lam_np1), _ptr(lam_n), float(dt),
                                                _stream(stream)), "dg_adjoint_step")
        return lam_n

    def dg_tape_len(self) -> int:
        return int(load().dg_tape_len(self.ctx))

    def dg_step_tape(self, w, dt: float, tape, stream=None):
        """One SSP-RK3 step of w in place, recording its stages and traces into tape."""
        _check(self.ctx, load().dg_step_tape(self.ctx, _ptr(w), float(dt), _ptr(tape), _stream(stream)),
               "dg_step_tape")
        return w

    def dg_adjoint_step_tape(self, w_n, tape, lam_np1, dt: float, lam_n=None, stream=None):
        import torch
        if lam_n is None:
            lam_n = torch.empty_like(w_n)
        _check(self.ctx, load().dg_adjoint_step_tape(self.ctx, _ptr(w_n), _ptr(tape), _ptr(lam_np1), _ptr(lam_n),
                                                     float(dt), _stream(stream)), "dg_adjoint_step_tape")
        return lam_n

    def dg_adjoint_segment(self, w_start, m: int, dt: float, states, tapes, lam, stream=None):
        """One checkpoint segment of a reverse sweep: m taped steps from w_start (states: (m + 1)
        state rows, tapes: m tape rows, both contiguous float64 CUDA buffers), then lam <- the
        transpose of the segment's Jacobian applied to lam, in place."""
        _check(self.ctx, load().dg_adjoint_segment(self.ctx, _ptr(w_start), int(m), float(dt), _ptr(states),
                                                   _ptr(tapes), _ptr(lam), _stream(stream)), "dg_adjoint_segment")
        return lam

    def dg_reinit(self, w, niter: int = 50, nu: float = 0.0, dtau: float = 0.0, stream=None):
        """Re-initialise the level set of w in place (end of Sec. 3; nu, dtau <= 0: defaults)."""
        _check(self.ctx, load().dg_reinit(self.ctx, _ptr(w), int(niter), float(nu), float(dtau), _stream(stream)),
               "dg_reinit")
        return w

    def dg_diag(self, w, stream=None):
        out = (ctypes.c_double * 16)()
        _check(self.ctx, load().dg_diag(self.ctx, _ptr(w), out, _stream(stream)), "dg_diag")
        return list(out)

    def dg_status_read(self, stream=None):
        return load().dg_status_read(self.ctx, _stream(stream))

    def dg_time_kernels(self, w, nrep=20, stream=None):
        out = (ctypes.c_double * 8)()
        n = load().dg_time_kernels(self.ctx, _ptr(w), int(nrep), out, 8, _stream(stream))
        if n < 0:
            raise DGError(-2, "dg_time_kernels failed")
        return list(out)[:n]

    def dg_step_launches(self, nsteps: int = 1) -> int:
        """Kernel launches of one dg_step call of nsteps steps (dg_step_launches)."""
        n = load().dg_step_launches(self.ctx, int(nsteps))
        if n < 0:
            raise DGError(-1, "dg_step_launches failed")
        return n

    def dg_kernel_costs(self):
        f = (ctypes.c_double * 8)()
        b = (ctypes.c_double * 8)()
        n = load().dg_kernel_costs(self.ctx, f, b, 8)
        return list(f)[:n], list(b)[:n]


class BatchSolver:
    """Many independent 2D problems advanced together (wraps a batch ``dg_ctx``, FP32-bulk).

    ``problems`` is a list of :class:`workloads.Workload`; ``dg_batch_step`` takes a list of
    float64 CUDA state tensors (one per problem) and a list of step sizes.
    """

    def __init__(self, problems, precision: str = "fp32bulk", tile: int = 0):
        """tile: 0 tunes the tile of every order on the first step; 1..4 fixes variant tile - 1."""
        lib = load()
        n = len(problems)
        meshes = (dg_mesh * n)()
        eoss = (dg_eos * n)()
        ps = (ctypes.c_int * n)()
        G = (ctypes.c_double * n)()
        E = (ctypes.c_double * n)()
        opts = None
        for k, pb in enumerate(problems):
            kw = pb.problem_kwargs()
            ps[k] = kw.pop("p")
            G[k], E[k] = kw.pop("Gamma"), kw.pop("eps")
            m, e, o = make_structs(precision=precision, check_finite=False, **kw)
            meshes[k], eoss[k] = m, e
            opts = o if opts is None else opts
        opts.batch_tile = int(tile)
        self._keep = (meshes, eoss, ps, G, E, opts)
        h = ctypes.c_void_p()
        st = lib.dg_batch_create(n, meshes, ps, eoss, G, E, ctypes.byref(opts), ctypes.byref(h))
        _check(None, st, "dg_batch_create")
        self.ctx = h
        self.n = n

    def close(self):
        if getattr(self, "ctx", None):
            load().dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dg_batch_step(self, ws, dts, nsteps: int, stream=None):
        ptrs = (ctypes.c_void_p * self.n)(*[_ptr(w).value for w in ws])
        dt = (ctypes.c_double * self.n)(*[float(x) for x in dts])
        _check(self.ctx, load().dg_batch_step(self.ctx, ptrs, dt, int(nsteps), _stream(stream)), "dg_batch_step")
        return ws

    def dg_batch_tiles(self):
        """Tiles chosen by the tuner (after the first dg_batch_step): one dict per order."""
        m = 8
        p, epb, minb = (ctypes.c_int * m)(), (ctypes.c_int * m)(), (ctypes.c_int * m)()
        best, dflt = (ctypes.c_double * m)(), (ctypes.c_double * m)()
        n = load().dg_batch_tiles(self.ctx, p, epb, minb, best, dflt, m)
        if n < 0:
            raise DGError(-1, "dg_batch_tiles: not a batch context")
        return [{"p": p[i], "epb": epb[i], "minb": minb[i], "ms": best[i], "ms_default_tile": dflt[i]}
                for i in range(n)]


ELEM = {"quad": 0, "tri": 1}


def _kin_mesh(problem) -> dg_mesh:
    m = dg_mesh()
    m.dim, m.nx, m.ny = 2, problem.nx, problem.ny
    m.x0, m.x1, m.y0, m.y1 = problem.x0, problem.x1, problem.y0, problem.y1
    for i in range(4):
        m.bc[i] = BC["periodic"]
    m.elem = ELEM[getattr(problem, "elem", "quad")]
    return m


def dg_kin_nodes(problem):
    """Node coordinates (x, y) of a kinematic-mode problem's state, from the library
    (``dg_kin_nodes``): float64 numpy arrays of N = 2 nx ny (p+1)(p+2)/2 nodes on triangles,
    nx ny (p+1)^2 on rectangles."""
    import numpy as np
    p = problem.p
    per = (p + 1) * (p + 2) // 2 * 2 if getattr(problem, "elem", "quad") == "tri" else (p + 1) ** 2
    N = problem.nx * problem.ny * per
    x, y = np.zeros(N), np.zeros(N)
    m = _kin_mesh(problem)
    dpt = ctypes.POINTER(ctypes.c_double)
    _check(None, load().dg_kin_nodes(ctypes.byref(m), p, x.ctypes.data_as(dpt), y.ctypes.data_as(dpt)),
           "dg_kin_nodes")
    return x, y


class KinematicSolver:
    """Kinematic mode (Sec. 4.1): phi and psi advected by a prescribed velocity, classical RK4
    (wraps a ``dg_kin_create`` context).  ``problem`` is a :class:`workloads.KinWorkload`; states
    are float64 CUDA tensors of shape (2, N)."""

    def __init__(self, problem):
        lib = load()
        m = _kin_mesh(problem)
        v = dg_velocity()
        v.kind, v.u0, v.v0, v.T = VEL[problem.vel], problem.u0, problem.v0, problem.T
        v.xc, v.yc = problem.xc, problem.yc
        self._keep = (m, v)
        h = ctypes.c_void_p()
        st = lib.dg_kin_create(ctypes.byref(m), problem.p, problem.Gamma, problem.eps, ctypes.byref(v),
                               problem.c_ip, ctypes.byref(h))
        _check(None, st, "dg_kin_create")
        self.ctx = h
        self.len = lib.dg_state_len(h)

    def close(self):
        if getattr(self, "ctx", None):
            load().dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dg_kin_rhs(self, w, t: float, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(w)
        _check(self.ctx, load().dg_kin_rhs(self.ctx, _ptr(w), float(t), _ptr(out), _stream(stream)), "dg_kin_rhs")
        return out

    def dg_kin_step(self, w, t0: float, dt: float, nsteps: int, stream=None):
        _check(self.ctx, load().dg_kin_step(self.ctx, _ptr(w), float(t0), float(dt), int(nsteps), _stream(stream)),
               "dg_kin_step")
        return w

    def dg_reinit(self, w, niter: int = 50, nu: float = 0.0, dtau: float = 0.0, stream=None):
        """Re-initialise the level set of w in place (end of Sec. 3; nu, dtau <= 0: defaults)."""
        _check(self.ctx, load().dg_reinit(self.ctx, _ptr(w), int(niter), float(nu), float(dtau), _stream(stream)),
               "dg_reinit")
        return w

    def dg_status_read(self, stream=None):
        return load().dg_status_read(self.ctx, _stream(stream))

