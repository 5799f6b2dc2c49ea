// Triangle kinematic-mode kernels (dg_tri.cuh) of orders 1..4 and their
// reference tables.
#include <cmath>

#include "dg_tri.cuh"

namespace dgpf {

template <int P>
static TriKernels tri_set() {
  return {&launch_tri_stage<P>, &launch_tri_velocity_table<P>, (const void *)&k_tri_stage<P>, TriGeom<P>::THREADS,
          TriGeom<P>::NQV + TriGeom<P>::NQE};
}

bool tri_kernels(int p, TriKernels *out) {
  switch (p) {
    case 1: *out = tri_set<1>(); return true;
    case 2: *out = tri_set<2>(); return true;
    case 3: *out = tri_set<3>(); return true;
    case 4: *out = tri_set<4>(); return true;
    default: return false;
  }
}

void tri_constants(double hx, double hy, double eta_tri, TriConst tc[2]) {
  for (int type = 0; type < 2; ++type) {
    const double v[3][2] = {{0.0, 0.0}, {hx, type == 0 ? 0.0 : hy}, {type == 0 ? hx : 0.0, hy}};
    TriConst &g = tc[type];
    const double xr = 0.5 * (v[1][0] - v[0][0]), yr = 0.5 * (v[1][1] - v[0][1]);
    const double xs = 0.5 * (v[2][0] - v[0][0]), ys = 0.5 * (v[2][1] - v[0][1]);
    g.det = xr * ys - xs * yr;
    g.idet = 1.0 / g.det;
    g.rx = ys / g.det;
    g.ry = -xs / g.det;
    g.sx = -yr / g.det;
    g.sy = xr / g.det;
    for (int f = 0; f < 3; ++f) {
      const int fn = (f + 1) % 3;
      const double dx = v[fn][0] - v[f][0], dy = v[fn][1] - v[f][1], len = std::sqrt(dx * dx + dy * dy);
      g.m0[f] = dy / len;
      g.m1[f] = -dx / len;
      g.hl[f] = 0.5 * len;
      g.ihl[f] = 2.0 / len;
      g.eta[f] = eta_tri / (2.0 * (2.0 * g.det) / len);  // h_e = 2 |T| / |e|, |T| = 2 det
      g.gr[f] = g.rx * g.m0[f] + g.ry * g.m1[f];
      g.gs[f] = g.sx * g.m0[f] + g.sy * g.m1[f];
    }
  }
}

int tri_group(int p) {
  switch (p) {
    case 1: return TriGeom<1>::EPB;
    case 2: return TriGeom<2>::EPB;
    case 3: return TriGeom<3>::EPB;
    case 4: return TriGeom<4>::EPB;
    default: return 0;
  }
}

namespace {

// n-point Gauss-Legendre rule on [-1, 1], ascending: Newton iteration on P_n
// from the Chebyshev points, P_n and P_n' by the three-term recurrence.
void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * n)), dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, pc = z;
      for (int k = 2; k <= n; ++k) {
        const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
        pm = pc;
        pc = pn;
      }
      dp = n * (z * pc - pm) / (z * z - 1.0);
      const double step = pc / dp;
      z -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    double pm = 1.0, pc = z;
    for (int k = 2; k <= n; ++k) {
      const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
      pm = pc;
      pc = pn;
    }
    dp = n * (z * pc - pm) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// A_m(lambda) = prod_{q<m} (p lambda - q) / (q + 1) and its derivative: the
// one-dimensional factor of the equispaced Lagrange basis in barycentric form.
void silvester(int p, int m, double lam, double *a, double *da) {
  double v = 1.0, d = 0.0;
  for (int q = 0; q < m; ++q) {
    const double f = (p * lam - q) / (q + 1.0), df = p / (q + 1.0);
    d = d * f + v * df;
    v *= f;
  }
  *a = v;
  *da = d;
}

// Nodal basis at (r, s): node (i, j) (j-major, i + j <= p) at (-1 + 2i/p,
// -1 + 2j/p) is l = A_i(l2) A_j(l3) A_k(l1), k = p - i - j, with the
// barycentric coordinates l1 = -(r + s)/2, l2 = (1 + r)/2, l3 = (1 + s)/2.
void basis(int p, double r, double s, double *l, double *lr, double *ls) {
  const double l1 = -0.5 * (r + s), l2 = 0.5 * (1.0 + r), l3 = 0.5 * (1.0 + s);
  int n = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i, ++n) {
      const int k = p - i - j;
      double a2, d2, a3, d3, a1, d1;
      silvester(p, i, l2, &a2, &d2);
      silvester(p, j, l3, &a3, &d3);
      silvester(p, k, l1, &a1, &d1);
      l[n] = a2 * a3 * a1;
      lr[n] = 0.5 * (d2 * a3 * a1 - a2 * a3 * d1);
      ls[n] = 0.5 * (a2 * d3 * a1 - a2 * a3 * d1);
    }
}

// Inverse of a symmetric positive definite n x n matrix by Cholesky; false if
// the matrix is not positive definite.
bool spd_inverse(int n, const std::vector<double> &A, std::vector<double> &Ai) {
  std::vector<double> Lc(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= Lc[j * n + k] * Lc[j * n + k];
    if (!(d > 0.0)) return false;
    Lc[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= Lc[i * n + k] * Lc[j * n + k];
      Lc[i * n + j] = v / Lc[j * n + j];
    }
  }
  Ai.assign(n * n, 0.0);
  std::vector<double> y(n), x(n);
  for (int c = 0; c < n; ++c) {  // solve L L^T x = e_c
    for (int i = 0; i < n; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= Lc[i * n + k] * y[k];
      y[i] = v / Lc[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < n; ++k) v -= Lc[k * n + i] * x[k];
      x[i] = v / Lc[i * n + i];
    }
    for (int i = 0; i < n; ++i) Ai[i * n + c] = x[i];
  }
  return true;
}

}  // namespace

std::vector<double> tri_tables(int p, const TriConst tc[2]) {
  if (p < 1 || p > 4) return {};
  const TriLayout L(p);
  std::vector<double> t(L.size(), 0.0), gx, gw;
  gauss_rule(L.NQ1, gx, gw);
  // Volume rule: the collapsed map r = (1 + a)(1 - b)/2 - 1, s = b of the
  // square onto the triangle, weight w_a w_b (1 - b)/2; q = b-index NQ1 + a-index.
  for (int ib = 0; ib < L.NQ1; ++ib)
    for (int ia = 0; ia < L.NQ1; ++ia) {
      const int q = ib * L.NQ1 + ia;
      const double a = gx[ia], b = gx[ib];
      const double r = 0.5 * (1.0 + a) * (1.0 - b) - 1.0, s = b;
      t[L.rv() + q] = r;
      t[L.sv() + q] = s;
      t[L.wv() + q] = gw[ia] * gw[ib] * 0.5 * (1.0 - b);
      basis(p, r, s, &t[L.bv() + q * L.NP], &t[L.brv() + q * L.NP], &t[L.bsv() + q * L.NP]);
    }
  // Edge points: parameter gx[k] along edge f from its first vertex to its second.
  std::vector<double> l(L.NP), lr(L.NP), ls(L.NP);
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < L.NQ1; ++k) {
      const int fk = f * L.NQ1 + k;
      const double u = gx[k];
      const double r = f == 0 ? u : (f == 1 ? -u : -1.0);
      const double s = f == 0 ? -1.0 : (f == 1 ? u : -u);
      t[L.re() + fk] = r;
      t[L.se() + fk] = s;
      basis(p, r, s, l.data(), lr.data(), ls.data());
      for (int m = 0; m <= p; ++m) {  // d/dt along the edge: (dr/dt, ds/dt) = (1, 0), (-1, 1), (0, -1)
        const int n = tri_edge_node(p, f, m);
        t[L.bev() + fk * L.P1 + m] = l[n];
        t[L.bet() + fk * L.P1 + m] = f == 0 ? lr[n] : (f == 1 ? -lr[n] + ls[n] : -ls[n]);
      }
      for (int type = 0; type < 2; ++type) {
        const TriConst &g = tc[type];
        for (int n = 0; n < L.NP; ++n)
          t[L.bn() + (type * L.NQE + fk) * L.NP + n] =
              (lr[n] * g.rx + ls[n] * g.sx) * g.m0[f] + (lr[n] * g.ry + ls[n] * g.sy) * g.m1[f];
      }
    }
  for (int k = 0; k < L.NQ1; ++k) t[L.we() + k] = gw[k];
  // Reference mass matrix sum_q w_q l_i l_j (exact: degree 2p <= 2 NQ1 - 2) and its inverse.
  std::vector<double> M(L.NP * L.NP, 0.0), Mi;
  for (int q = 0; q < L.NQV; ++q)
    for (int i = 0; i < L.NP; ++i)
      for (int j = 0; j < L.NP; ++j)
        M[i * L.NP + j] += t[L.wv() + q] * t[L.bv() + q * L.NP + i] * t[L.bv() + q * L.NP + j];
  if (!spd_inverse(L.NP, M, Mi)) return {};
  for (int i = 0; i < L.NP * L.NP; ++i) t[L.minv() + i] = Mi[i];
  return t;
}

}  // namespace dgpf
