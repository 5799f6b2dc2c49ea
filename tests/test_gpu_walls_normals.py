"""GPU parity on the states that pin the oracle's wall and degenerate-normal branches
(tests/test_oracle_walls.py), for the FP64 path (1e-12 of the oracle's scale S) and the
FP32-bulk path (2e-6 of S plus the FP32 storage bound), and the device's non-physical flag.

* slip channel with a flow crossing the walls, viscous stress on;
* plane Poiseuille flow between no-slip walls (viscous, gravity);
* a constant level-set patch (|grad psi| = 0: n = 0) with exact pure-phase regions
  (phi = 0 and phi = 1 exactly, where phi (1 - phi) = 0);
* 1D: a slab between a no-slip wall and the Riemann-invariant pressure boundary;
* the FP32 normal cut-off: FP32 kernels set n = 0 where |grad psi| < 1e-4 (below that the
  direction of a distance-like psi stored in FP32 is noise), the oracle and the FP64 kernels
  where |grad psi| < 1e-12.  On a level set that is not a distance the two differ by the
  sharpening flux Gamma phi (1 - phi) n of the affected nodes, which the test bounds.
"""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import problem
from tests.test_gpu_fp32bulk import TOL32, _storage_bound
from tests.test_gpu_parity import _assert_parity, _rhs_both

pytestmark = pytest.mark.gpu


def _slip_channel_crossing_flow():
    wl = W.Workload(name="slipch", dim=2, nx=5, ny=4, p=3, bc=("periodic", "periodic", "slip", "slip"),
                    Gamma=1.0, eps=0.05, viscous=True, mu=(2e-3, 5e-3))
    x, y = W.node_coords(wl)
    u = 0.4 + 0.3 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
    v = 0.25 - 0.2 * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    # the drop's distance taken periodically in x, so that no field jumps at the periodic seam
    s = W.periodic_distance(x, y, 0.45, 0.55) - 0.2
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5, u, v)
    return wl


def _poiseuille(p=3):
    mu, g = 0.05, 0.4
    wl = W.Workload(name="pois", dim=2, nx=3, ny=5, p=p, bc=("periodic", "periodic", "noslip", "noslip"),
                    gamma=(1.4, 1.4), pinf=(0.0, 0.0), rho0=(1.0, 1.0), mu=(mu, mu), viscous=True,
                    gravity=True, g=(g, 0.0), Gamma=0.3, eps=0.02)
    x, y = W.node_coords(wl)
    # a level set with a gradient everywhere: with a constant one the transport rate of psi is pure
    # rounding of D applied to a constant, at which scale the two codes' summation orders differ
    psi = 0.2 * np.sin(2 * np.pi * x) + 0.1 * y
    wl.w = W.conserved(wl, np.full(wl.N, 0.5), psi, 1e5, g * y * (1 - y) / (2 * mu), 0.0)
    return wl


def _degenerate_normals(p=3):
    """A drop whose level set is constant in the elements of the lower-left quarter (n = 0
    there), with phi exactly 0 and exactly 1 in whole elements."""
    wl = W.Workload(name="degen", dim=2, nx=6, ny=6, p=p, Gamma=1.0, eps=0.04)
    x, y = W.node_coords(wl)
    s = np.hypot(x - 0.55, y - 0.6) - 0.22
    phi = W.tanh_profile(s, wl.eps)
    e = np.repeat(np.arange(wl.E), wl.Np)
    ex, ey = e % wl.nx, e // wl.nx
    phi = np.where(ex == 5, 1.0, phi)             # a pure phase-1 column
    phi = np.where((ex == 0) & (ey == 5), 0.0, phi)  # a pure phase-2 element
    psi = np.where((ex < 3) & (ey < 3), 0.3, s)   # constant level set: |grad psi| = 0
    wl.w = W.conserved(wl, phi, psi, 1e5, 0.6, -0.3)
    return wl


def _slab_1d_walls(p=3):
    """1D: a water slab in air between a no-slip wall (x = 0) and the pressure boundary (x = 1,
    P_b = 1.2e5 against P = 1e5 inside), with a flow toward the pressure side."""
    wl = W.Workload(name="slab1d_walls", dim=1, nx=9, ny=1, p=p, bc=("noslip", "pressure", "periodic", "periodic"),
                    p_bc=(0.0, 1.2e5, 0.0, 0.0), Gamma=1.0)
    wl.eps = wl.hx
    x, _ = W.node_coords(wl)
    s = 0.2 - np.abs(x - 0.55)
    u = 0.5 * np.sin(np.pi * x)
    wl.w = W.conserved(wl, W.tanh_profile(s, wl.eps), s, 1e5 + 50.0 * x, u, 0.0)
    return wl


CASES = {"slip_channel": _slip_channel_crossing_flow, "poiseuille_p3": lambda: _poiseuille(3),
         "poiseuille_p2": lambda: _poiseuille(2), "degenerate_normals": _degenerate_normals,
         "slab_1d_walls_p3": lambda: _slab_1d_walls(3), "slab_1d_walls_p5": lambda: _slab_1d_walls(5)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_rhs_parity(orc, dg, case):
    _assert_parity(*_rhs_both(orc, dg, CASES[case]()))


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32bulk_rhs_parity(orc, dg, case):
    import torch
    wl = CASES[case]()
    L_ref, S = orc.rhs(problem(orc, wl), wl.w, want_scale=True)
    s = dg.Solver(wl, precision="fp32bulk")
    L = s.dg_rhs(torch.from_numpy(np.array(wl.w)).cuda()).cpu().numpy()
    assert s.dg_status_read() == 0
    s.close()
    extra = _storage_bound(orc, wl, wl.w)
    for v in range(7):
        sc = S[v].max()
        if sc == 0:
            continue
        err = np.abs(L[v] - L_ref[v]).max()
        assert err <= TOL32 * sc + extra.get(v, 0.0), (v, err / sc)


def test_fp32_normal_cutoff_bound(orc, dg):
    """psi = c (x + y / 2) with |grad psi| = 5.6e-5: a unit normal for the oracle and the FP64
    kernels, n = 0 for the FP32 kernels.  The FP32 phase-field rate differs from the oracle's by
    at most the divergence and the face jumps of the missing sharpening flux,
    Gamma max phi (1 - phi) (2 (2/h) max_i sum_c |D_ic| + 2 / (w_0 h)), and does differ (the
    cut-off is active); the FP64 kernels keep parity with the oracle."""
    import torch
    wl = W.Workload(name="cut", dim=2, nx=6, ny=6, p=3, Gamma=1.0, eps=0.04)
    x, y = W.node_coords(wl)
    s = np.hypot(x - 0.5, y - 0.5) - 0.25
    phi = W.tanh_profile(s, wl.eps)
    psi = 5e-5 * (x + 0.5 * y)
    w = W.conserved(wl, phi, psi, 1e5, 0.0, 0.0)
    pb = problem(orc, wl)
    L_ref, S = orc.rhs(pb, w, want_scale=True)
    s32 = dg.Solver(wl, precision="fp32bulk")
    L32 = s32.dg_rhs(torch.from_numpy(w.copy()).cuda()).cpu().numpy()
    s32.close()
    xi, wt = orc.gll(wl.p)
    D = orc.lagrange_deriv(wl.p, xi)
    h = min(wl.hx, wl.hy)
    sharp = wl.Gamma * np.max(phi * (1 - phi))
    bound = sharp * ((2.0 / h) * np.abs(D).sum(axis=1).max() * 2 + 2.0 / (wt[-1] * h))
    diff = np.abs(L32[0] - L_ref[0])
    assert diff.max() <= bound + TOL32 * S[0].max()
    assert diff.max() > 1e3 * TOL32 * S[0].max()  # the cut-off is active here
    # the FP64 kernels keep the unit normal: parity with the oracle
    _assert_parity(*_rhs_both(orc, dg, wl, w))


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
@pytest.mark.parametrize("fault", ["negative_density", "negative_pressure"])
def test_nonphysical_flag(dg, precision, fault):
    """A state with rho <= 0 at one node, or with P + Pinf_mix <= 0 (rho E far below the
    stiffened-gas constant), latches DG_ERR_NONPHYSICAL; the flag is cleared by the read."""
    import torch
    wl = W.drop_2d(n=4, p=3, seed=1)
    w = wl.w.copy()
    n = 37
    if fault == "negative_density":
        w[2, n] = -abs(w[2, n]) - 1.0
        w[3, n] = 0.0
    else:
        w[6, n] = -1e9  # rho e < 0: P (1 + den) + Cm = (rho e (1 + den) - Cm) / den < 0
    s = dg.Solver(wl, precision=precision)
    s.dg_rhs(torch.from_numpy(w).cuda())
    assert s.dg_status_read() == -6
    assert s.dg_status_read() == 0
    # a physical state raises nothing
    s.dg_rhs(torch.from_numpy(wl.w.copy()).cuda())
    assert s.dg_status_read() == 0
    s.close()
