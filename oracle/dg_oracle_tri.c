/*
 * dg_oracle_tri.c -- plain FP64 CPU oracle of the kinematic mode (Sec. 4.1) on
 * triangular elements (the paper's mesh (b), Sec. 4.1, Rider-Kothe test).
 *
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.c); shares no code with the CUDA
 * library.
 *
 * Discretisation (readings of what the paper leaves open, also listed in the
 * design notes):
 *   - mesh: each cell of an nx x ny Cartesian grid of the periodic rectangle is
 *     split along its rising diagonal into a lower-right triangle (type A,
 *     vertices (x_i, y_j), (x_i+1, y_j), (x_i+1, y_j+1)) and an upper-left one
 *     (type B, vertices (x_i, y_j), (x_i+1, y_j+1), (x_i, y_j+1)); element index
 *     2 (i + nx j) + type, counter-clockwise vertices v1, v2, v3;
 *   - reference triangle (-1,-1), (1,-1), (-1,1); x = v1 + (1+r)/2 (v2 - v1) +
 *     (1+s)/2 (v3 - v1); edges 0: v1->v2, 1: v2->v3, 2: v3->v1;
 *   - nodal Lagrange basis of degree p on the equispaced nodes
 *     (r, s) = (-1 + 2i/p, -1 + 2j/p), i + j <= p, ordered j-major;
 *   - no collocation: volume integrals with the collapsed Gauss-Legendre rule
 *     of (p+2)^2 points (r = (1+a)(1-b)/2 - 1, s = b, weight (1-b)/2), edge
 *     integrals with p+2 Gauss-Legendre points, a full element mass matrix;
 *   - the velocity is the analytical field evaluated at the quadrature points;
 *   - SIP penalty eta = c_ip (p+1)(p+2) / h_e, h_e = 2 |T| / |e|;
 *   - everything else as the phi and psi rows of the quadrilateral scheme:
 *     transport flux (lambda - m.u-) [[f]], lambda = max(|u-.m|, |u+.m|), SIP
 *     flux of a_1 with its symmetric term, classical RK4.
 */
#include "dg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TMAXP 4
#define TMAXNP 15   /* (TMAXP+1)(TMAXP+2)/2 */
#define TMAXQ 6     /* TMAXP + 2 */

/* Legendre P_n and its derivative by the three-term recurrence. */
static void leg(int n, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;  /* P_k' = P_{k-2}' + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

/* n-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n). */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      leg(n, z, &P, &dP);
      double dz = P / dP;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double P, dP;
    leg(n, z, &P, &dP);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

/* Reference element data of order p. */
typedef struct {
  int p, Np, nq, Nq;                 /* nodes, 1D rule size, volume points */
  double rn[TMAXNP], sn[TMAXNP];     /* nodes */
  double Vinv[TMAXNP * TMAXNP];      /* inverse Vandermonde of the modal basis at the nodes */
  double qr[TMAXQ * TMAXQ], qs[TMAXQ * TMAXQ], qw[TMAXQ * TMAXQ];  /* volume rule */
  double gx[TMAXQ], gw[TMAXQ];       /* 1D Gauss-Legendre rule (edges) */
} tref_t;

/* Modal basis: Legendre products P_i(r) P_j(s), i + j <= p (spans P_p). */
static void modal(int p, double r, double s, double *phi, double *dr, double *ds) {
  double Pr[TMAXP + 1], dPr[TMAXP + 1], Ps[TMAXP + 1], dPs[TMAXP + 1];
  for (int k = 0; k <= p; ++k) {
    leg(k, r, &Pr[k], &dPr[k]);
    leg(k, s, &Ps[k], &dPs[k]);
  }
  int m = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i, ++m) {
      phi[m] = Pr[i] * Ps[j];
      if (dr) dr[m] = dPr[i] * Ps[j];
      if (ds) ds[m] = Pr[i] * dPs[j];
    }
}

/* Gauss-Jordan inverse of an n x n matrix (partial pivoting); returns 0 on success. */
static int invert(int n, const double *A, double *Ainv) {
  double a[TMAXNP * 2 * TMAXNP];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(a[i * 2 * n + c]) > fabs(a[piv * 2 * n + c])) piv = i;
    if (a[piv * 2 * n + c] == 0.0) return -1;
    for (int j = 0; j < 2 * n; ++j) {
      double t = a[c * 2 * n + j];
      a[c * 2 * n + j] = a[piv * 2 * n + j];
      a[piv * 2 * n + j] = t;
    }
    double d = a[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) a[c * 2 * n + j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      double f = a[i * 2 * n + c];
      for (int j = 0; j < 2 * n; ++j) a[i * 2 * n + j] -= f * a[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = a[i * 2 * n + n + j];
  return 0;
}

static int tref_init(tref_t *t, int p) {
  if (p < 1 || p > TMAXP) return -1;
  t->p = p;
  t->Np = (p + 1) * (p + 2) / 2;
  t->nq = p + 2;
  t->Nq = t->nq * t->nq;
  int m = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i, ++m) {
      t->rn[m] = -1.0 + 2.0 * i / p;
      t->sn[m] = -1.0 + 2.0 * j / p;
    }
  double V[TMAXNP * TMAXNP];
  for (int n = 0; n < t->Np; ++n) modal(p, t->rn[n], t->sn[n], &V[n * t->Np], NULL, NULL);
  if (invert(t->Np, V, t->Vinv)) return -1;
  gauss_legendre(t->nq, t->gx, t->gw);
  for (int ia = 0; ia < t->nq; ++ia)
    for (int ib = 0; ib < t->nq; ++ib) {
      double a = t->gx[ia], b = t->gx[ib];
      int q = ib * t->nq + ia;
      t->qr[q] = 0.5 * (1.0 + a) * (1.0 - b) - 1.0;
      t->qs[q] = b;
      t->qw[q] = t->gw[ia] * t->gw[ib] * 0.5 * (1.0 - b);
    }
  return 0;
}

/* Nodal basis values l_n and reference derivatives at (r, s): l = V^-T modal. */
static void nodal(const tref_t *t, double r, double s, double *l, double *lr, double *ls) {
  double ph[TMAXNP], dr[TMAXNP], ds[TMAXNP];
  modal(t->p, r, s, ph, dr, ds);
  for (int n = 0; n < t->Np; ++n) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < t->Np; ++k) {
      double vi = t->Vinv[k * t->Np + n];  /* l_n = sum_k (V^-1)_{kn} phi_k */
      a += vi * ph[k];
      b += vi * dr[k];
      c += vi * ds[k];
    }
    l[n] = a;
    if (lr) lr[n] = b;
    if (ls) ls[n] = c;
  }
}

/* Reference (r, s) of the point at parameter t in [-1, 1] along edge f. */
static void edge_point(int f, double t, double *r, double *s) {
  switch (f) {
    case 0: *r = t; *s = -1.0; break;             /* v1 (-1,-1) -> v2 (1,-1) */
    case 1: *r = -t; *s = t; break;               /* v2 (1,-1) -> v3 (-1,1) */
    default: *r = -1.0; *s = -t; break;           /* v3 (-1,1) -> v1 (-1,-1) */
  }
}

/* ------------------------------------------------------------------------ */
/* Mesh                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  double v[3][2];        /* counter-clockwise vertices */
  double det;            /* d(x,y)/d(r,s) */
  double rx, ry, sx, sy; /* inverse map derivatives */
} tgeo_t;

static int tri_check(const orc_problem *pr) {
  if (!pr || pr->dim != 2 || pr->nx < 1 || pr->ny < 1 || pr->p < 1 || pr->p > TMAXP) return -1;
  if (!(pr->x1 > pr->x0) || !(pr->y1 > pr->y0)) return -1;
  return 0;
}

static void tri_geo(const orc_problem *pr, int e, tgeo_t *g) {
  int cell = e / 2, type = e % 2;
  int ci = cell % pr->nx, cj = cell / pr->nx;
  double hx = (pr->x1 - pr->x0) / pr->nx, hy = (pr->y1 - pr->y0) / pr->ny;
  double x0 = pr->x0 + ci * hx, y0 = pr->y0 + cj * hy;
  g->v[0][0] = x0; g->v[0][1] = y0;
  if (type == 0) {
    g->v[1][0] = x0 + hx; g->v[1][1] = y0;
    g->v[2][0] = x0 + hx; g->v[2][1] = y0 + hy;
  } else {
    g->v[1][0] = x0 + hx; g->v[1][1] = y0 + hy;
    g->v[2][0] = x0; g->v[2][1] = y0 + hy;
  }
  double xr = 0.5 * (g->v[1][0] - g->v[0][0]), yr = 0.5 * (g->v[1][1] - g->v[0][1]);
  double xs = 0.5 * (g->v[2][0] - g->v[0][0]), ys = 0.5 * (g->v[2][1] - g->v[0][1]);
  g->det = xr * ys - xs * yr;
  g->rx = ys / g->det;
  g->ry = -xs / g->det;
  g->sx = -yr / g->det;
  g->sy = xr / g->det;
}

static void tri_map(const tgeo_t *g, double r, double s, double *x, double *y) {
  *x = g->v[0][0] + 0.5 * (1.0 + r) * (g->v[1][0] - g->v[0][0]) + 0.5 * (1.0 + s) * (g->v[2][0] - g->v[0][0]);
  *y = g->v[0][1] + 0.5 * (1.0 + r) * (g->v[1][1] - g->v[0][1]) + 0.5 * (1.0 + s) * (g->v[2][1] - g->v[0][1]);
}

/* Neighbour of element e across its edge f and the neighbour's edge index. */
static int tri_neighbour(const orc_problem *pr, int e, int f, int *f2) {
  int cell = e / 2, type = e % 2;
  int ci = cell % pr->nx, cj = cell / pr->nx, nx = pr->nx, ny = pr->ny;
  if (type == 0) {
    if (f == 0) { *f2 = 1; return 2 * (ci + nx * ((cj + ny - 1) % ny)) + 1; }  /* bottom -> B below, top */
    if (f == 1) { *f2 = 2; return 2 * ((ci + 1) % nx + nx * cj) + 1; }         /* right -> B right, left */
    *f2 = 0; return 2 * cell + 1;                                               /* diagonal -> B, diagonal */
  }
  if (f == 0) { *f2 = 2; return 2 * cell; }                                      /* diagonal -> A, diagonal */
  if (f == 1) { *f2 = 0; return 2 * (ci + nx * ((cj + 1) % ny)); }               /* top -> A above, bottom */
  *f2 = 1; return 2 * ((ci + nx - 1) % nx + nx * cj);                            /* left -> A left, right */
}

long orc_tri_num_nodes(const orc_problem *pr) {
  if (tri_check(pr)) return -1;
  return 2L * pr->nx * pr->ny * ((pr->p + 1) * (pr->p + 2) / 2);
}

int orc_tri_nodes(const orc_problem *pr, double *x, double *y) {
  tref_t t;
  if (tri_check(pr) || tref_init(&t, pr->p)) return -1;
  int E = 2 * pr->nx * pr->ny;
  for (int e = 0; e < E; ++e) {
    tgeo_t g;
    tri_geo(pr, e, &g);
    for (int n = 0; n < t.Np; ++n) tri_map(&g, t.rn[n], t.sn[n], &x[(long)e * t.Np + n], &y[(long)e * t.Np + n]);
  }
  return 0;
}

/* Integral of a nodal field f over the domain. */
int orc_tri_integral(const orc_problem *pr, const double *f, double *out) {
  tref_t t;
  if (tri_check(pr) || tref_init(&t, pr->p)) return -1;
  int E = 2 * pr->nx * pr->ny;
  double acc = 0.0;
  for (int e = 0; e < E; ++e) {
    tgeo_t g;
    tri_geo(pr, e, &g);
    for (int q = 0; q < t.Nq; ++q) {
      double l[TMAXNP], v = 0.0;
      nodal(&t, t.qr[q], t.qs[q], l, NULL, NULL);
      for (int n = 0; n < t.Np; ++n) v += l[n] * f[(long)e * t.Np + n];
      acc += t.qw[q] * g.det * v;
    }
  }
  *out = acc;
  return 0;
}

/* Values of the element's phi and psi, gradients, normal n = grad psi/|grad psi|
   and a_1 at reference point (r, s). */
typedef struct {
  double phi, psi, gphi[2], gpsi[2], n[2], a1[2], a1m[2];
} tpt_t;

static void tri_eval(const orc_problem *pr, const tref_t *t, const tgeo_t *g, const double *phi,
                     const double *psi, double r, double s, tpt_t *o, double *l, double *gl) {
  double lr[TMAXNP], ls[TMAXNP];
  nodal(t, r, s, l, lr, ls);
  memset(o, 0, sizeof(*o));
  for (int n = 0; n < t->Np; ++n) {
    gl[2 * n] = lr[n] * g->rx + ls[n] * g->sx;
    gl[2 * n + 1] = lr[n] * g->ry + ls[n] * g->sy;
    o->phi += l[n] * phi[n];
    o->psi += l[n] * psi[n];
    for (int d = 0; d < 2; ++d) {
      o->gphi[d] += gl[2 * n + d] * phi[n];
      o->gpsi[d] += gl[2 * n + d] * psi[n];
    }
  }
  double norm = sqrt(o->gpsi[0] * o->gpsi[0] + o->gpsi[1] * o->gpsi[1]);
  double sp = o->phi * (1.0 - o->phi);
  for (int d = 0; d < 2; ++d) {
    o->n[d] = norm < 1e-12 ? 0.0 : o->gpsi[d] / norm;
    o->a1[d] = pr->Gamma * (pr->eps * o->gphi[d] - sp * o->n[d]);
    o->a1m[d] = pr->Gamma * (fabs(pr->eps * o->gphi[d]) + fabs(sp * o->n[d]));
  }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side and RK4                                                  */
/* ------------------------------------------------------------------------ */

int orc_tri_rhs(const orc_problem *pr, const orc_velocity *vel, double t, const double *w, double *L, double *S) {
  tref_t T;
  if (tri_check(pr) || !vel || tref_init(&T, pr->p)) return -1;
  const int Np = T.Np, E = 2 * pr->nx * pr->ny;
  const long N = (long)E * Np;
  const double Gam = pr->Gamma, eps = pr->eps;
  const double *phi = w, *psi = w + N;
  double *R = (double *)calloc((size_t)2 * N, sizeof(double));
  double *A = (double *)calloc((size_t)2 * N, sizeof(double));
  if (!R || !A) {
    free(R); free(A);
    return -2;
  }
  for (int e = 0; e < E; ++e) {
    tgeo_t g;
    tri_geo(pr, e, &g);
    const long base = (long)e * Np;
    double *Rp = R + base, *Rs = R + N + base, *Ap = A + base, *As = A + N + base;
    /* 1. Volume: int grad l_n . (-a_1) - int l_n u . grad phi, and - int l_n u . grad psi. */
    for (int q = 0; q < T.Nq; ++q) {
      tpt_t o;
      double l[TMAXNP], gl[2 * TMAXNP], x, y, u, v;
      tri_eval(pr, &T, &g, phi + base, psi + base, T.qr[q], T.qs[q], &o, l, gl);
      tri_map(&g, T.qr[q], T.qs[q], &x, &y);
      orc_velocity_at(vel, x, y, t, &u, &v);
      double wq = T.qw[q] * g.det;
      double tp = u * o.gphi[0] + v * o.gphi[1], ts = u * o.gpsi[0] + v * o.gpsi[1];
      double tpm = fabs(u * o.gphi[0]) + fabs(v * o.gphi[1]), tsm = fabs(u * o.gpsi[0]) + fabs(v * o.gpsi[1]);
      for (int n = 0; n < Np; ++n) {
        Rp[n] += wq * (-(gl[2 * n] * o.a1[0] + gl[2 * n + 1] * o.a1[1]) - l[n] * tp);
        Ap[n] += wq * (fabs(gl[2 * n]) * o.a1m[0] + fabs(gl[2 * n + 1]) * o.a1m[1] + fabs(l[n]) * tpm);
        Rs[n] += -wq * l[n] * ts;
        As[n] += wq * fabs(l[n]) * tsm;
      }
    }
    /* 2. Edges: transport (lambda - m.u-) [[f]], SIP flux of a_1 and its symmetric term. */
    for (int f = 0; f < 3; ++f) {
      int f2;
      int e2 = tri_neighbour(pr, e, f, &f2);
      tgeo_t g2;
      tri_geo(pr, e2, &g2);
      const double *P = g.v[f], *Q = g.v[(f + 1) % 3];
      double dx = Q[0] - P[0], dy = Q[1] - P[1], len = sqrt(dx * dx + dy * dy);
      double m[2] = {dy / len, -dx / len};
      double he = 2.0 * (2.0 * g.det) / len;              /* 2 |T| / |e|, |T| = 2 det */
      double eta = pr->c_ip * (pr->p + 1.0) * (pr->p + 2.0) / he;
      for (int k = 0; k < T.nq; ++k) {
        double r, s, r2, s2, x, y, x2, y2, u, v, u2, v2;
        edge_point(f, T.gx[k], &r, &s);
        edge_point(f2, -T.gx[k], &r2, &s2);
        tpt_t om, op;
        double l[TMAXNP], gl[2 * TMAXNP], l2[TMAXNP], gl2[2 * TMAXNP];
        tri_eval(pr, &T, &g, phi + base, psi + base, r, s, &om, l, gl);
        tri_eval(pr, &T, &g2, phi + (long)e2 * Np, psi + (long)e2 * Np, r2, s2, &op, l2, gl2);
        tri_map(&g, r, s, &x, &y);
        tri_map(&g2, r2, s2, &x2, &y2);
        orc_velocity_at(vel, x, y, t, &u, &v);
        orc_velocity_at(vel, x2, y2, t, &u2, &v2);
        double wf = T.gw[k] * 0.5 * len;
        double unm = u * m[0] + v * m[1], unp = u2 * m[0] + v2 * m[1];
        double lam = fmax(fabs(unm), fabs(unp));
        double jump = op.phi - om.phi, hjs = 0.5 * (op.psi - om.psi);
        double gn = 0.5 * ((op.gphi[0] + om.gphi[0]) * m[0] + (op.gphi[1] + om.gphi[1]) * m[1]);
        double sp = op.phi * (1.0 - op.phi), sm = om.phi * (1.0 - om.phi);
        double sharp = 0.5 * (sp * (op.n[0] * m[0] + op.n[1] * m[1]) + sm * (om.n[0] * m[0] + om.n[1] * m[1]));
        double ahat = Gam * (eps * (gn + eta * jump) - sharp);
        double amag = Gam * (eps * (0.5 * (fabs(op.gphi[0] * m[0] + op.gphi[1] * m[1]) +
                                           fabs(om.gphi[0] * m[0] + om.gphi[1] * m[1])) + fabs(eta * jump)) +
                             0.5 * (fabs(sp) + fabs(sm)));
        double fphi = (lam - unm) * 0.5 * jump + ahat;
        double fmag = fabs(lam * 0.5 * jump) + fabs(unm * 0.5 * jump) + amag;
        double sym = 0.5 * Gam * eps * jump;
        for (int n = 0; n < Np; ++n) {
          double glm = gl[2 * n] * m[0] + gl[2 * n + 1] * m[1];
          Rp[n] += wf * (l[n] * fphi - sym * glm);
          Ap[n] += wf * (fabs(l[n]) * fmag + fabs(sym * glm));
          Rs[n] += wf * l[n] * (lam - unm) * hjs;
          As[n] += wf * fabs(l[n]) * (fabs(lam * hjs) + fabs(unm * hjs));
        }
      }
    }
  }
  /* 3. L = M^-1 R with the element mass matrix M_ij = int l_i l_j (the same rule). */
  double M[TMAXNP * TMAXNP] = {0}, Mi[TMAXNP * TMAXNP];
  for (int q = 0; q < T.Nq; ++q) {
    double l[TMAXNP];
    nodal(&T, T.qr[q], T.qs[q], l, NULL, NULL);
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j) M[i * Np + j] += T.qw[q] * l[i] * l[j];
  }
  if (invert(Np, M, Mi)) {
    free(R); free(A);
    return -3;
  }
  for (int e = 0; e < E; ++e) {
    tgeo_t g;
    tri_geo(pr, e, &g);
    for (int v = 0; v < 2; ++v) {
      const long base = (long)v * N + (long)e * Np;
      for (int i = 0; i < Np; ++i) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Np; ++j) {
          a += Mi[i * Np + j] * R[base + j];
          b += fabs(Mi[i * Np + j]) * A[base + j];
        }
        L[base + i] = a / g.det;
        if (S) S[base + i] = b / g.det;
      }
    }
  }
  free(R);
  free(A);
  return 0;
}

int orc_tri_rk4(const orc_problem *pr, const orc_velocity *vel, double *w, double t0, double dt, int nsteps) {
  long N = orc_tri_num_nodes(pr);
  if (N < 0 || nsteps < 0) return -1;
  size_t len = (size_t)2 * N;
  double *k = (double *)malloc(len * sizeof(double));
  double *acc = (double *)malloc(len * sizeof(double));
  double *ws = (double *)malloc(len * sizeof(double));
  if (!k || !acc || !ws) {
    free(k); free(acc); free(ws);
    return -2;
  }
  int rc = 0;
  for (int st = 0; st < nsteps && rc == 0; ++st) {
    double t = t0 + st * dt;
    rc = orc_tri_rhs(pr, vel, t, w, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] = k[i]; ws[i] = w[i] + 0.5 * dt * k[i]; }
    if (rc == 0) rc = orc_tri_rhs(pr, vel, t + 0.5 * dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] += 2.0 * k[i]; ws[i] = w[i] + 0.5 * dt * k[i]; }
    if (rc == 0) rc = orc_tri_rhs(pr, vel, t + 0.5 * dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] += 2.0 * k[i]; ws[i] = w[i] + dt * k[i]; }
    if (rc == 0) rc = orc_tri_rhs(pr, vel, t + dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) w[i] = w[i] + dt / 6.0 * (acc[i] + k[i]);
  }
  free(k); free(acc); free(ws);
  return rc;
}

/* Mass matrix M_ij = int_T l_i l_j of element e (row-major Np x Np). */
int orc_tri_mass(const orc_problem *pr, int e, double *M) {
  tref_t T;
  if (tri_check(pr) || tref_init(&T, pr->p) || e < 0 || e >= 2 * pr->nx * pr->ny) return -1;
  tgeo_t g;
  tri_geo(pr, e, &g);
  memset(M, 0, sizeof(double) * T.Np * T.Np);
  for (int q = 0; q < T.Nq; ++q) {
    double l[TMAXNP];
    nodal(&T, T.qr[q], T.qs[q], l, NULL, NULL);
    for (int i = 0; i < T.Np; ++i)
      for (int j = 0; j < T.Np; ++j) M[i * T.Np + j] += T.qw[q] * g.det * l[i] * l[j];
  }
  return 0;
}
