"""CPU-side checks of the C ABI: the library builds/loads, exports every function
declared in include/dgpf.h, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_05002_gb300 import build
    build.build()
    import paper_2306_05002_gb300 as pkg
    return pkg.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 8
    for name in declared:
        assert hasattr(lib, name), name
    import paper_2306_05002_gb300 as pkg
    assert sorted(pkg.EXPORTS) == sorted(n for n in declared if n in pkg.EXPORTS)
    for name in declared:
        assert name in pkg.EXPORTS, f"{name} declared but not bound in Python"


def _args(**over):
    import paper_2306_05002_gb300 as pkg
    kw = dict(dim=2, nx=4, ny=4, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=("periodic",) * 4,
              gamma=(1.4, 4.4), pinf=(0.0, 6e8), rho0=(1.0, 1000.0))
    p = over.pop("p", 3)
    Gamma = over.pop("Gamma", 1.0)
    eps = over.pop("eps", 0.01)
    kw.update(over)
    m, e, o = pkg.make_structs(**kw)
    return m, p, e, Gamma, eps, o


@pytest.mark.parametrize("over,code", [
    (dict(dim=3), -1),
    (dict(p=0), -7),
    (dict(p=9), -7),
    (dict(nx=0), -1),
    (dict(dim=1, ny=2), -1),
    (dict(x1=0.0), -1),
    (dict(bc=("periodic", "noslip", "periodic", "periodic")), -1),
    (dict(bc=("noslip", "noslip", "noslip", "pressure"), p_bc=(0.0, 0.0, 0.0, float("nan"))), -1),
    (dict(gamma=(1.0, 1.4)), -1),
    (dict(Gamma=-1.0), -1),
])
def test_create_rejects_invalid_arguments(lib, over, code):
    m, p, e, Gamma, eps, o = _args(**over)
    h = ctypes.c_void_p(123)
    st = lib.dg_create(ctypes.byref(m), p, ctypes.byref(e), Gamma, eps, ctypes.byref(o), ctypes.byref(h))
    assert st == code
    assert h.value is None
    assert lib.dg_last_error(None)  # a message is available


def test_null_context_is_safe(lib):
    assert lib.dg_state_len(None) == 0
    assert lib.dg_rhs(None, None, None, None) == -1
    assert lib.dg_step(None, None, 1.0, 1, None) == -1
    assert lib.dg_step_host(None, None, 1.0, 1, None) == -1
    assert lib.dg_batch_tiles(None, None, None, None, None, None, 4) == -1
    assert lib.dg_step_launches(None, 1) == -1
    lib.dg_destroy(None)
    assert isinstance(lib.dg_last_error(None), bytes)


def test_batch_create_rejects_unsupported_forms(lib):
    """Checked before any device work: FP64 and viscous batches are not provided."""
    import paper_2306_05002_gb300 as pkg
    m, p, e, Gamma, eps, o = _args()
    meshes = (pkg.dg_mesh * 1)(m)
    eoss = (pkg.dg_eos * 1)(e)
    ps = (ctypes.c_int * 1)(p)
    G = (ctypes.c_double * 1)(Gamma)
    E = (ctypes.c_double * 1)(eps)
    h = ctypes.c_void_p()
    o.prec = 0
    assert lib.dg_batch_create(1, meshes, ps, eoss, G, E, ctypes.byref(o), ctypes.byref(h)) == -7
    o.prec, o.viscous = 1, 1
    assert lib.dg_batch_create(1, meshes, ps, eoss, G, E, ctypes.byref(o), ctypes.byref(h)) == -7
    o.viscous, o.batch_tile = 0, 5
    assert lib.dg_batch_create(1, meshes, ps, eoss, G, E, ctypes.byref(o), ctypes.byref(h)) == -1
    assert h.value is None


def _kin_args(**over):
    import paper_2306_05002_gb300 as pkg
    m = pkg.dg_mesh()
    m.dim, m.nx, m.ny = over.pop("dim", 2), over.pop("nx", 4), over.pop("ny", 4)
    m.x0, m.x1, m.y0, m.y1 = -0.5, 0.5, -0.5, 0.5
    m.elem = over.pop("elem", 0)
    bc = over.pop("bc", ("periodic",) * 4)
    for i in range(4):
        m.bc[i] = pkg.BC[bc[i]]
    v = pkg.dg_velocity()
    v.kind, v.u0, v.v0, v.T = over.pop("kind", 1), 0.0, 0.0, over.pop("T", 4.0)
    return m, over.pop("p", 3), over.pop("Gamma", 1.0), over.pop("eps", 0.05), v


@pytest.mark.parametrize("over,code", [
    (dict(dim=1, ny=1), -1),
    (dict(p=0), -7),
    (dict(bc=("periodic", "periodic", "noslip", "noslip")), -7),
    (dict(kind=7), -1),
    (dict(T=0.0), -1),
    (dict(Gamma=-1.0), -1),
    (dict(elem=2), -1),
    (dict(elem=1, p=5), -7),
    (dict(nx=1 << 14, ny=(1 << 12) + 1), -1),              # more than 2^26 cells
    (dict(nx=1 << 13, ny=1 << 13, p=5), -1),               # 2^26 cells of 36 nodes: 2.4e9 nodes
    (dict(nx=1 << 13, ny=(1 << 13) + 1, p=4, elem=1), -1),  # more than 2^26 cells of triangles
])
def test_kin_create_rejects_invalid_arguments(lib, over, code):
    m, p, G, eps, v = _kin_args(**over)
    h = ctypes.c_void_p(123)
    assert lib.dg_kin_create(ctypes.byref(m), p, G, eps, ctypes.byref(v), 1.0, ctypes.byref(h)) == code
    assert h.value is None


def test_kin_calls_reject_other_contexts(lib):
    assert lib.dg_kin_rhs(None, None, 0.0, None, None) == -1
    assert lib.dg_kin_step(None, None, 0.0, 1.0, 1, None) == -1


def test_reinit_rejects_null_and_negative_arguments(lib):
    assert lib.dg_reinit(None, None, 1, 0.0, 0.0, None) == -1


def test_create_rejects_problems_beyond_the_node_limit(lib):
    """7 N doubles must be indexable with 32-bit node counts: 16384^2 p5 elements are refused during
    argument checking, before any device call."""
    import paper_2306_05002_gb300 as pkg
    m, eos, o = pkg.make_structs(2, 1 << 14, 1 << 14, 0.0, 1.0, 0.0, 1.0, ("periodic",) * 4, (4.4, 1.4),
                                 (6e8, 0.0), (1000.0, 1.0))
    h = ctypes.c_void_p(123)
    assert lib.dg_create(ctypes.byref(m), 5, ctypes.byref(eos), 1.0, 0.05, ctypes.byref(o), ctypes.byref(h)) == -1
    assert h.value is None


def test_full_model_rejects_triangles(lib):
    import paper_2306_05002_gb300 as pkg
    m, eos, o = pkg.make_structs(2, 4, 4, 0.0, 1.0, 0.0, 1.0, ("periodic",) * 4, (4.4, 1.4), (6e8, 0.0),
                                 (1000.0, 1.0))
    m.elem = 1
    h = ctypes.c_void_p(123)
    assert lib.dg_create(ctypes.byref(m), 3, ctypes.byref(eos), 1.0, 0.05, ctypes.byref(o), ctypes.byref(h)) == -7
    assert h.value is None


@pytest.mark.parametrize("elem,p", [("tri", 1), ("tri", 3), ("tri", 4), ("quad", 2), ("quad", 5)])
def test_kin_nodes_match_oracle_and_workload(lib, orc, elem, p):
    """dg_kin_nodes (host code of the library) against the oracle's and the input generator's node
    coordinates: the state layout the three share."""
    import numpy as np
    import paper_2306_05002_gb300 as pkg
    from paper_2306_05002_gb300 import workloads as W
    wl = W.KinWorkload(name="t", nx=3, ny=2, p=p, x0=-0.3, x1=0.9, y0=0.1, y1=0.7, elem=elem)
    x, y = pkg.dg_kin_nodes(wl)
    pb = orc.Problem(**wl.problem_kwargs())
    xo, yo = orc.tri_nodes(pb) if elem == "tri" else orc.nodes(pb)
    xw, yw = W._kin_nodes(wl)
    assert len(x) == wl.N == len(xo)
    assert np.abs(x - xo).max() < 1e-15 and np.abs(y - yo).max() < 1e-15
    assert np.abs(x - xw).max() < 1e-15 and np.abs(y - yw).max() < 1e-15


def test_kin_nodes_rejects_invalid_arguments(lib):
    import numpy as np
    m, _, _, _, _ = _kin_args(elem=1)
    x = np.zeros(1000)
    dpt = ctypes.POINTER(ctypes.c_double)
    assert lib.dg_kin_nodes(None, 3, x.ctypes.data_as(dpt), x.ctypes.data_as(dpt)) == -1
    assert lib.dg_kin_nodes(ctypes.byref(m), 3, None, x.ctypes.data_as(dpt)) == -1
    assert lib.dg_kin_nodes(ctypes.byref(m), 5, x.ctypes.data_as(dpt), x.ctypes.data_as(dpt)) == -7
    m.elem = 3
    assert lib.dg_kin_nodes(ctypes.byref(m), 3, x.ctypes.data_as(dpt), x.ctypes.data_as(dpt)) == -1


def test_noalloc_rejects_triangles_before_gpu_work(lib):
    """The allocation-free right-hand side covers the rectangles only: a triangle mesh is refused
    during argument checking, before any device call."""
    import paper_2306_05002_gb300 as pkg
    m, eos, o = pkg.make_structs(2, 4, 4, 0.0, 1.0, 0.0, 1.0, ("periodic",) * 4, (4.4, 1.4), (6e8, 0.0),
                                 (1000.0, 1.0))
    m.elem = 1
    f = lib.dg_rhs_noalloc
    f.argtypes = [ctypes.POINTER(pkg.dg_mesh), ctypes.c_int, ctypes.POINTER(pkg.dg_eos), ctypes.c_double,
                  ctypes.c_double, ctypes.POINTER(pkg.dg_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(m), 3, ctypes.byref(eos), 1.0, 0.05, ctypes.byref(o), 16, 4096, None) == -7
    m.elem = 2
    assert f(ctypes.byref(m), 3, ctypes.byref(eos), 1.0, 0.05, ctypes.byref(o), 16, 4096, None) == -1



def test_peak_probe_rejects_invalid_arguments(lib):
    """Checked before any GPU work."""
    import ctypes
    out = ctypes.c_double()
    assert lib.dg_peak_flops(2, 100, ctypes.byref(out), None) == -1
    assert lib.dg_peak_flops(0, 0, ctypes.byref(out), None) == -1
    assert lib.dg_peak_flops(0, 100, None, None) == -1
