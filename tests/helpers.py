"""Small helpers shared by the tests (no DG arithmetic here)."""
import numpy as np

from paper_2306_05002_gb300 import workloads as W


def problem(orc, wl):
    return orc.Problem(**wl.problem_kwargs())


def mass_weights(orc, wl):
    """Diagonal of the collocated mass matrix, one entry per node (w_i w_j J)."""
    _, wt = orc.gll(wl.p)
    if wl.dim == 2:
        Mn = np.outer(wt, wt).reshape(-1) * (wl.hx * wl.hy / 4.0)
    else:
        Mn = wt * (wl.hx / 2.0)
    return np.tile(Mn, wl.E)


def uniform_state(wl, phi, P, u, v, psi=0.0):
    n = wl.N
    return W.conserved(wl, np.full(n, phi, dtype=float), np.full(n, psi, dtype=float), P, u, v)


def rel_err(a, b, scale):
    """max |a - b| / max scale  (scale: the oracle's rounding scale S)."""
    s = np.max(np.abs(scale))
    return np.max(np.abs(a - b)) / (s if s > 0 else 1.0)
