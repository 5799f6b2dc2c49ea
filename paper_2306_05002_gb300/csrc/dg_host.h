// dg_host.h -- host-side set-up shared by every entry point of libdgpf that
// describes one problem: argument validation, the Gauss-Lobatto-Legendre
// operator tables of Sec. 3 and the kernels' parameter block.  Everything here
// writes into caller-provided storage (no heap, no device calls), so the
// allocation-free entry point uses the same code as dg_create.
#pragma once

#include <cmath>

#include "dg_common.cuh"
#include "dgpf.h"

namespace dgpf {

constexpr int HOST_MAXP1 = 6;  // orders up to 5

// GLL nodes by Newton's method on (1 - x^2) P_p'(x), written with the
// identity (1 - x^2) P_p' = p (P_{p-1} - x P_p) and the Newton step
// x <- x - (x P_p - P_{p-1}) / ((p+1) P_p); weights 2 / (p (p+1) P_p(x)^2).
// x and w hold p + 1 values.
inline void gll_nodes_into(int p, double *x, double *w) {
  for (int i = 0; i <= p; ++i) x[i] = -std::cos(M_PI * i / p);
  auto legendre = [p](double t, double *Pp, double *Pm) {
    double a = 1.0, b = t;  // P_0, P_1
    for (int k = 2; k <= p; ++k) {
      const double c = ((2.0 * k - 1.0) * t * b - (k - 1.0) * a) / k;
      a = b;
      b = c;
    }
    *Pp = b;
    *Pm = a;
  };
  for (int it = 0; it < 200; ++it) {
    double moved = 0.0;
    for (int i = 1; i < p; ++i) {
      double Pp, Pm;
      legendre(x[i], &Pp, &Pm);
      const double dx = (x[i] * Pp - Pm) / ((p + 1.0) * Pp);
      x[i] -= dx;
      moved = std::fmax(moved, std::fabs(dx));
    }
    if (moved < 1e-16) break;
  }
  for (int i = 0; i <= p / 2; ++i) {  // exact symmetry about 0
    const double s = 0.5 * (x[p - i] - x[i]);
    x[i] = -s;
    x[p - i] = s;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
  for (int i = 0; i <= p; ++i) {
    double Pp = 1.0, Pm;
    if (i != 0 && i != p) legendre(x[i], &Pp, &Pm);
    w[i] = 2.0 / (p * (p + 1.0) * Pp * Pp);
  }
}

// Lagrange derivative matrix D[a][b] = l_b'(x_a) from barycentric weights
// (n nodes, D holds n * n values).
inline void lagrange_derivative_into(int n, const double *x, double *D) {
  double lam[HOST_MAXP1 + 2];
  for (int j = 0; j < n; ++j) {
    lam[j] = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (x[j] - x[k]);
  }
  for (int a = 0; a < n; ++a) {
    double diag = 0.0;
    for (int b = 0; b < n; ++b) {
      if (b == a) continue;
      D[a * n + b] = (lam[b] / lam[a]) / (x[a] - x[b]);
      diag -= D[a * n + b];
    }
    D[a * n + a] = diag;
  }
}

// Operator table (OpsLayout, OpsLayout{p+1, Np}.size() doubles) for one
// element size: (2/h) D, (2/h) Dhat with Dhat = W^-1 D^T W, the GLL weights,
// the inverse of the collocated mass matrix and the face quadrature weights.
inline void build_ops_into(int dim, int p, double hx, double hy, double *ops) {
  const int P1 = p + 1, Np = dim == 2 ? P1 * P1 : P1;
  const double J = dim == 2 ? 0.25 * hx * hy : 0.5 * hx;
  double xi[HOST_MAXP1], wt[HOST_MAXP1], D[HOST_MAXP1 * HOST_MAXP1];
  gll_nodes_into(p, xi, wt);
  lagrange_derivative_into(P1, xi, D);
  const OpsLayout L{P1, Np};
  for (int t = 0; t < L.size(); ++t) ops[t] = 0.0;
  const double rx = 2.0 / hx, ry = 2.0 / hy;
  for (int a = 0; a < P1; ++a)
    for (int b = 0; b < P1; ++b) {
      ops[L.Dx() + a * P1 + b] = rx * D[a * P1 + b];
      ops[L.Dy() + a * P1 + b] = ry * D[a * P1 + b];
      const double dh = wt[b] * D[b * P1 + a] / wt[a];
      ops[L.Dhx() + a * P1 + b] = rx * dh;
      ops[L.Dhy() + a * P1 + b] = ry * dh;
    }
  for (int a = 0; a < P1; ++a) ops[L.wt() + a] = wt[a];
  for (int a = 0; a < Np; ++a) {
    const double wa = dim == 2 ? wt[a % P1] * wt[a / P1] : wt[a];
    ops[L.invM() + a] = 1.0 / (wa * J);
  }
  for (int k = 0; k < P1; ++k) {
    ops[L.wfx() + k] = dim == 2 ? wt[k] * 0.5 * hy : 1.0;
    ops[L.wfy() + k] = dim == 2 ? wt[k] * 0.5 * hx : 1.0;
  }
}

// Validation of one problem of the two-phase model: NULL when valid, else the
// reason, with *code the status to return.
inline const char *check_problem(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                                 dg_status *code) {
  *code = DG_ERR_ARG;
  if (!mesh || !eos) return "mesh and eos are required";
  if (mesh->dim != 1 && mesh->dim != 2) return "dim must be 1 or 2";
  if (mesh->elem != DG_ELEM_QUAD) {
    *code = mesh->elem == DG_ELEM_TRI ? DG_ERR_UNSUPPORTED : DG_ERR_ARG;
    return "the two-phase flow model runs on rectangular elements only (elem = DG_ELEM_QUAD)";
  }
  if (p < 1 || p > 5) {
    *code = DG_ERR_UNSUPPORTED;
    return "order p must be in 1..5";
  }
  if (mesh->nx < 1 || mesh->ny < 1 || (mesh->dim == 1 && mesh->ny != 1)) return "bad element counts (1D needs ny = 1)";
  if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0))) return "empty domain";
  for (int f = 0; f < 4; ++f)
    if (mesh->bc[f] < DG_BC_PERIODIC || mesh->bc[f] > DG_BC_PRESSURE) return "unknown boundary condition";
  for (int f = 0; f < 4; ++f)
    if (mesh->bc[f] == DG_BC_PRESSURE && !std::isfinite(mesh->p_bc[f])) return "pressure boundary needs a finite p_bc";
  if ((mesh->bc[0] == DG_BC_PERIODIC) != (mesh->bc[1] == DG_BC_PERIODIC) ||
      (mesh->dim == 2 && (mesh->bc[2] == DG_BC_PERIODIC) != (mesh->bc[3] == DG_BC_PERIODIC)))
    return "periodic sides must be paired";
  for (int l = 0; l < 2; ++l)
    if (!(eos->gamma[l] > 1.0) || !(eos->rho0[l] > 0.0) || eos->mu[l] < 0.0) return "need gamma > 1, rho0 > 0, mu >= 0";
  if (!(Gamma >= 0.0) || !(eps >= 0.0)) return "need Gamma, eps >= 0";
  const long long Np = mesh->dim == 2 ? (long long)(p + 1) * (p + 1) : p + 1;
  if ((long long)mesh->nx * mesh->ny * Np * 7 >= (1LL << 31)) return "problem too large for one context";
  *code = DG_OK;
  return nullptr;
}

// Options with the defaults filled in (FP64, c_ip = 1 when not positive).
inline dg_opts normalised_opts(const dg_opts *opts) {
  dg_opts o{};
  o.prec = DG_FP64;
  o.c_ip = 1.0;
  if (opts) o = *opts;
  if (o.c_ip <= 0.0) o.c_ip = 1.0;
  return o;
}

// Kernel parameters of one problem.  The closure constants are computed with
// the same expressions as the stiffened-gas formula of Sec. 2 so that the
// pressure is reproducible.  ops and status are left for the caller.
inline Params make_params(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps, const dg_opts &o,
                          double hx, double hy) {
  const int P1 = p + 1, Np = mesh->dim == 2 ? P1 * P1 : P1;
  Params q{};
  q.nx = mesh->nx;
  q.ny = mesh->ny;
  q.E = mesh->nx * mesh->ny;
  q.N = q.E * Np;
  for (int f = 0; f < 4; ++f) {
    q.bc[f] = mesh->bc[f];
    q.p_bc[f] = mesh->bc[f] == DG_BC_PRESSURE ? mesh->p_bc[f] : 0.0;
  }
  q.C1 = eos->gamma[0] * eos->pinf[0] / (eos->gamma[0] - 1.0);
  q.C2 = eos->gamma[1] * eos->pinf[1] / (eos->gamma[1] - 1.0);
  q.g1 = 1.0 / (eos->gamma[0] - 1.0);
  q.g2 = 1.0 / (eos->gamma[1] - 1.0);
  q.Bp = eos->gamma[0] / (eos->gamma[0] - 1.0) - eos->gamma[1] / (eos->gamma[1] - 1.0);
  q.dC = q.C1 - q.C2;
  q.rho01 = eos->rho0[0];
  q.rho02 = eos->rho0[1];
  q.drho0 = eos->rho0[0] - eos->rho0[1];
  q.mu1 = eos->mu[0];
  q.mu2 = eos->mu[1];
  q.sigma = eos->sigma;
  q.gx = eos->g[0];
  q.gy = eos->g[1];
  q.Gamma = Gamma;
  q.eps = eps;
  q.eta_x = o.c_ip * P1 * P1 / hx;
  q.eta_y = o.c_ip * P1 * P1 / hy;
  q.gravity = o.gravity != 0;
  q.check_finite = o.check_finite != 0;
  q.grad_lift = o.grad_lift != 0;
  return q;
}

}  // namespace dgpf
