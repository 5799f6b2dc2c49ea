"""Pins of the oracle's one-dimensional operators (Sec. 3: Lagrange basis on GLL nodes,
collocated quadrature) against closed forms and exact identities."""
import os

import numpy as np
import pytest
from numpy import sqrt  # noqa: F401  (used by the golden table expressions)

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_gll():
    rows = {}
    with open(os.path.join(HERE, "golden", "gll_lobatto_table.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            p, x, w = line.split()
            rows.setdefault(int(p), []).append((eval(x), eval(w)))
    return rows


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_closed_forms(orc, p):
    xi, wt = orc.gll(p)
    ref = _golden_gll()[p]
    np.testing.assert_allclose(xi, [r[0] for r in ref], rtol=0, atol=1e-15)
    np.testing.assert_allclose(wt, [r[1] for r in ref], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_quadrature_exact_to_degree_2p_minus_1(orc, p):
    xi, wt = orc.gll(p)
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(wt, xi ** k) - exact) < 1e-14
    # and not exact at degree 2p (Lobatto rules stop at 2p-1)
    assert abs(np.dot(wt, xi ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_derivative_exact_on_polynomials(orc, p):
    xi, _ = orc.gll(p)
    D = orc.lagrange_deriv(p, xi)
    for k in range(0, p + 1):
        f = xi ** k
        df = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ f, df, rtol=0, atol=1e-12 * max(1, k))


@pytest.mark.parametrize("p", range(1, 9))
def test_summation_by_parts(orc, p):
    """D^T W + W D = diag(-1, 0, ..., 0, 1) for collocated GLL quadrature."""
    xi, wt = orc.gll(p)
    D = orc.lagrange_deriv(p, xi)
    Wm = np.diag(wt)
    B = np.zeros((p + 1, p + 1))
    B[0, 0], B[p, p] = -1.0, 1.0
    np.testing.assert_allclose(D.T @ Wm + Wm @ D, B, rtol=0, atol=1e-13)
