/*
 * dg_oracle.c -- plain FP64 CPU oracle for the explicit DG right-hand side of
 * Tonicello & Ihme, "A high-order diffused-interface approach for two-phase
 * compressible flow simulations using a Discontinuous Galerkin framework"
 * (arXiv 2306.05002).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path.  It shares no
 * code with the CUDA library.
 *
 * What it computes, in the paper's order:
 *   - the system of Sec. 2 (phase field phi = phi_1, level set psi, partial
 *     densities m_l = rho_l phi_l, momentum, total energy) with
 *     a_1 = Gamma (eps grad phi - phi (1 - phi) n),  n = grad psi / |grad psi|,
 *     R_l = rho_l^(0) a_l,  f = R_1 + R_2,  k = |u|^2 / 2   (Sec. 2);
 *   - the stiffened-gas pressure, phasic enthalpies and mixture rules (Sec. 2);
 *   - the nodal DG weak form of Sec. 3 (eq. "weakDG") on Cartesian affine
 *     elements, tensor-product Lagrange basis on Gauss-Lobatto-Legendre (GLL)
 *     nodes, quadrature collocated at those nodes (so M is diagonal);
 *   - the quasi-conservative transport of phi and psi with the one-sided
 *     "tilde" and averaged "hat" fluxes of Sec. 3, Lax-Friedrichs fluxes for
 *     the conservative equations, and the symmetric interior penalty (SIP)
 *     flux for every a_l-derived term (Sec. 3);
 *   - viscous stress, gravity and CSF surface tension of Sec. 2;
 *   - three-stage SSP Runge-Kutta in time;
 *   - the kinematic mode of Sec. 4.1: phase field and level set alone,
 *     advected by a prescribed velocity (uniform, or the Rider-Kothe vortex),
 *     with the classical four-stage Runge-Kutta method in time;
 *   - the level-set re-initialisation of the end of Sec. 3, in pseudo-time.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes of the repository):
 *   - "-" is the element's own trace, "+" the neighbour's; [[q]] is the half
 *     jump (q+ - q-)/2 and {q} the average, exactly as printed in Sec. 3;
 *   - the characteristic speed c of the transport flux is the local
 *     Lax-Friedrichs speed lambda = max(|u-.m| + c-, |u+.m| + c+) with the
 *     mixture sound speed c^2 = gamma (P + Pinf) / rho from the mixture rules,
 *     and the same lambda is used in every equation;
 *   - rho_l^(0) is a constant reference density per phase;
 *   - the sharpening part phi(1-phi)n uses the central flux {phi(1-phi)n}.m,
 *     the diffusive part the SIP flux eps({grad phi}.m + eta (phi+ - phi-))
 *     with eta = c_ip (p+1)^2 / h and the symmetric term of the SIP bilinear
 *     form;
 *   - every other equation carries its a_1-derived term as a coefficient C_q
 *     times the phi-equation flux, with face averages {C_q} at faces:
 *       C_m1 = rho_1^(0), C_m2 = -rho_2^(0), C_rhou = (rho_1^(0)-rho_2^(0)) u,
 *       C_rhoE = B + (rho_1^(0)-rho_2^(0)) k,  B = rho_1 H_1 - rho_2 H_2;
 *   - n = 0 where |grad psi| < 1e-12;
 *   - gradients of phi and psi: broken (element-local) by default; with the
 *     option grad_lift, BR1-lifted (the broken gradient plus M^-1 times the
 *     face integrals of l ({f} - f-) m, the central trace), and those lifted
 *     gradients give a_1, the normal, the SIP flux's {grad phi} and the CSF
 *     delta; the non-conservative transport -u.grad(phi), -u.grad(psi) keeps
 *     the broken gradient (its face flux already carries the jump);
 *   - viscous flux: {tau}.m + eta {mu} (u+ - u-) for momentum and
 *     {tau.u}.m + eta {mu} (k+ - k-) for energy (no symmetric term);
 *   - walls: ghost state equal to the own state with the velocity (no-slip)
 *     or its normal component (slip) reversed; ghost gradients equal the own
 *     ones; no a_1 flux crosses a wall;
 *   - the Riemann-invariant boundary "with zero velocity and constant
 *     pressure" (Sec. 4.2): the exterior state of the boundary Riemann problem
 *     holds the own phi, psi and partial densities at rest at the prescribed
 *     pressure (rho E from the stiffened-gas relation), and the
 *     Lax-Friedrichs flux between the two states carries it in; gradients and
 *     a_1 are treated as at a wall;
 *   - kinematic mode: a uniform velocity is taken as given, the Rider-Kothe
 *     vortex as the discrete curl of its stream function interpolated at the
 *     nodes (discretely divergence-free, normal component continuous across
 *     faces, so the phase field's mass is conserved to round-off), and the
 *     characteristic speed of the transport flux is the advection speed alone,
 *     lambda = max(|u-.m|, |u+.m|) (there is no sound speed in the kinematic
 *     system); everything else is the phi and psi rows of the full scheme;
 *   - re-initialisation: the equation is taken as
 *       d(psi)/d(tau) = S (1 - |grad psi|) + div(nu grad psi),
 *     the sign with which |grad psi| relaxes to 1 (as printed, with
 *     "+ S (1 - |grad psi|)" on the left-hand side, |grad psi| moves away
 *     from 1 at the interface: a garbled sign); the smeared sign is evaluated
 *     once from psi0 and its broken gradient (S = sign(psi0) where
 *     |grad psi0| < 1e-12); its
 *     diffusion carries the same SIP flux and penalty as a_1, with no flux
 *     through walls; three-stage SSP Runge-Kutta in pseudo-time (the paper
 *     names no pseudo-time integrator).
 */
#include "dg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV ORC_NV
#define MAXP 8

/* Loops over elements (or nodes) whose iterations write only their own
   element's (or node's) entries: the OpenMP build (-fopenmp) runs them in
   parallel and computes bit-identical results; the plain build, the one the
   tests pin, is single-threaded. */
#ifdef _OPENMP
#include <omp.h>
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OMP_FOR
#endif

int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* One-dimensional operators                                                */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) and its derivative, by the three-term recurrence. */
static void legendre(int n, double x, double *Pn, double *dPn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *Pn = 1.0; *dPn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *Pn = p1;
  /* (1 - x^2) P_n' = n (P_{n-1} - x P_n); only used at interior points. */
  *dPn = n * (p0 - x * p1) / (1.0 - x * x);
}

int orc_gll(int p, double *xi, double *wt) {
  if (p < 1 || p > MAXP) return -1;
  /* End points plus the p-1 roots of P_p', found by Newton's method from
     Chebyshev-Gauss-Lobatto guesses. */
  xi[0] = -1.0;
  xi[p] = 1.0;
  for (int k = 1; k < p; ++k) {
    double x = -cos(M_PI * k / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, &P, &dP);
      /* P_p'' from the Legendre equation: (1-x^2) P'' = 2x P' - p(p+1) P */
      double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xi[k] = x;
  }
  /* Symmetrise (the nodes are symmetric about 0). */
  for (int k = 0; k <= p / 2; ++k) {
    double s = 0.5 * (xi[p - k] - xi[k]);
    xi[k] = -s;
    xi[p - k] = s;
  }
  if (p % 2 == 0) xi[p / 2] = 0.0;
  for (int k = 0; k <= p; ++k) {
    double P, dP;
    if (k == 0 || k == p) {
      P = 1.0; /* |P_p(+-1)| = 1 */
    } else {
      legendre(p, xi[k], &P, &dP);
    }
    wt[k] = 2.0 / (p * (p + 1.0) * P * P);
  }
  return 0;
}

/* Derivative of the b-th Lagrange polynomial through nodes xi, at x:
   l_b'(x) = sum_{k != b} 1/(xi_b - xi_k) prod_{m != b,k} (x - xi_m)/(xi_b - xi_m). */
static double lagrange_deriv_at(int p, const double *xi, int b, double x) {
  double s = 0.0;
  for (int k = 0; k <= p; ++k) {
    if (k == b) continue;
    double t = 1.0 / (xi[b] - xi[k]);
    for (int m = 0; m <= p; ++m) {
      if (m == b || m == k) continue;
      t *= (x - xi[m]) / (xi[b] - xi[m]);
    }
    s += t;
  }
  return s;
}

int orc_lagrange_deriv(int p, const double *xi, double *D) {
  if (p < 1 || p > MAXP) return -1;
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) D[a * (p + 1) + b] = lagrange_deriv_at(p, xi, b, xi[a]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Problem geometry                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_problem *pr;
  int dim, p, P1, Np, nx, ny, E;
  long N;
  double hx, hy, J;          /* element sizes and volume Jacobian */
  double xi[MAXP + 1], wt[MAXP + 1], D[(MAXP + 1) * (MAXP + 1)];
  double C[2], gi[2];        /* gamma_l Pinf_l/(gamma_l-1), 1/(gamma_l-1) */
} geo_t;

static int check_problem(const orc_problem *pr) {
  if (!pr) return -1;
  if (pr->dim != 1 && pr->dim != 2) return -1;
  if (pr->p < 1 || pr->p > MAXP) return -1;
  if (pr->nx < 1 || pr->ny < 1) return -1;
  if (pr->dim == 1 && pr->ny != 1) return -1;
  if (!(pr->x1 > pr->x0)) return -1;
  if (pr->dim == 2 && !(pr->y1 > pr->y0)) return -1;
  for (int f = 0; f < 4; ++f)
    if (pr->bc[f] < ORC_BC_PERIODIC || pr->bc[f] > ORC_BC_PRESSURE) return -1;
  if ((pr->bc[0] == ORC_BC_PERIODIC) != (pr->bc[1] == ORC_BC_PERIODIC)) return -1;
  if (pr->dim == 2 && (pr->bc[2] == ORC_BC_PERIODIC) != (pr->bc[3] == ORC_BC_PERIODIC)) return -1;
  for (int l = 0; l < 2; ++l)
    if (!(pr->gamma[l] > 1.0)) return -1;
  return 0;
}

static int geo_init(geo_t *g, const orc_problem *pr) {
  if (check_problem(pr)) return -1;
  g->pr = pr;
  g->dim = pr->dim;
  g->p = pr->p;
  g->P1 = pr->p + 1;
  g->Np = pr->dim == 2 ? g->P1 * g->P1 : g->P1;
  g->nx = pr->nx;
  g->ny = pr->ny;
  g->E = pr->nx * pr->ny;
  g->N = (long)g->E * g->Np;
  g->hx = (pr->x1 - pr->x0) / pr->nx;
  g->hy = pr->dim == 2 ? (pr->y1 - pr->y0) / pr->ny : 1.0;
  g->J = pr->dim == 2 ? 0.25 * g->hx * g->hy : 0.5 * g->hx;
  orc_gll(g->p, g->xi, g->wt);
  orc_lagrange_deriv(g->p, g->xi, g->D);
  for (int l = 0; l < 2; ++l) {
    g->C[l] = pr->gamma[l] * pr->pinf[l] / (pr->gamma[l] - 1.0);
    g->gi[l] = 1.0 / (pr->gamma[l] - 1.0);
  }
  return 0;
}

long orc_num_nodes(const orc_problem *pr) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  return g.N;
}

/* Quadrature weight of node a (product of 1D GLL weights). */
static double node_weight(const geo_t *g, int a) {
  int i = a % g->P1, j = a / g->P1;
  return g->dim == 2 ? g->wt[i] * g->wt[j] : g->wt[i];
}

/* Gradient of the basis function l_b at node a of the same element. */
static void grad_basis(const geo_t *g, int b, int a, double gr[2]) {
  int bi = b % g->P1, bj = b / g->P1, ai = a % g->P1, aj = a / g->P1;
  gr[0] = (aj == bj) ? (2.0 / g->hx) * g->D[ai * g->P1 + bi] : 0.0;
  gr[1] = (g->dim == 2 && ai == bi) ? (2.0 / g->hy) * g->D[aj * g->P1 + bj] : 0.0;
}

int orc_nodes(const orc_problem *pr, double *x, double *y) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  for (int e = 0; e < g.E; ++e) {
    int ex = e % g.nx, ey = e / g.nx;
    for (int a = 0; a < g.Np; ++a) {
      int i = a % g.P1, j = a / g.P1;
      long n = (long)e * g.Np + a;
      x[n] = pr->x0 + g.hx * (ex + 0.5 * (g.xi[i] + 1.0));
      if (y) y[n] = g.dim == 2 ? pr->y0 + g.hy * (ey + 0.5 * (g.xi[j] + 1.0)) : 0.0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pointwise closure (Sec. 2)                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  double phi, psi, m1, m2, ru, rv, rE;
  double rho, u, v, k, P, c, B, mu;
} prim_t;

/* Stiffened-gas pressure from rho e and phi (Sec. 2), mixture sound speed
   from the mixture rules of Sec. 2, and B = rho_1 H_1 - rho_2 H_2 with
   rho_l H_l = gamma_l (P + Pinf_l) / (gamma_l - 1). */
static void closure(const geo_t *g, const double *wn, prim_t *q) {
  const orc_problem *pr = g->pr;
  q->phi = wn[ORC_PHI];
  q->psi = wn[ORC_PSI];
  q->m1 = wn[ORC_M1];
  q->m2 = wn[ORC_M2];
  q->ru = wn[ORC_RU];
  q->rv = wn[ORC_RV];
  q->rE = wn[ORC_RE];
  double phi1 = q->phi, phi2 = 1.0 - q->phi;
  q->rho = q->m1 + q->m2;
  q->u = q->ru / q->rho;
  q->v = q->rv / q->rho;
  q->k = 0.5 * (q->u * q->u + q->v * q->v);
  /* rho e = rho E - |rho u|^2 / (2 rho) */
  double rhoe = q->rE - 0.5 * (q->ru * q->ru + q->rv * q->rv) / q->rho;
  q->P = (rhoe - (phi1 * g->C[0] + phi2 * g->C[1])) / (phi1 * g->gi[0] + phi2 * g->gi[1]);
  /* mixture: 1/(gamma-1) = sum phi_l/(gamma_l-1); Pinf gamma/(gamma-1) = sum phi_l C_l */
  double Gm = phi1 * g->gi[0] + phi2 * g->gi[1];
  double Cm = phi1 * g->C[0] + phi2 * g->C[1];
  double gam = 1.0 + 1.0 / Gm;
  double pinf = Cm * (gam - 1.0) / gam;
  q->c = sqrt(gam * (q->P + pinf) / q->rho);
  q->B = pr->gamma[0] * (q->P + pr->pinf[0]) / (pr->gamma[0] - 1.0) -
         pr->gamma[1] * (q->P + pr->pinf[1]) / (pr->gamma[1] - 1.0);
  q->mu = pr->mu[0] * phi1 + pr->mu[1] * phi2;
}

int orc_primitives(const orc_problem *pr, const double *w, double *prim) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  for (long n = 0; n < g.N; ++n) {
    double wn[NV];
    for (int v = 0; v < NV; ++v) wn[v] = w[v * g.N + n];
    prim_t q;
    closure(&g, wn, &q);
    prim[0 * g.N + n] = q.rho;
    prim[1 * g.N + n] = q.u;
    prim[2 * g.N + n] = q.v;
    prim[3 * g.N + n] = q.P;
    prim[4 * g.N + n] = q.c;
    prim[5 * g.N + n] = q.B;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-node derived fields                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  prim_t q;
  double gphi[2], gpsi[2], gu[2], gv[2];
  double bphi[2], bpsi[2];  /* broken gradients of phi and psi (the transport term's) */
  double n[2];          /* interface normal from the level set */
  double a1[2], a1m[2]; /* a_1 and the magnitude of its two parts */
  double tau[2][2];     /* viscous stress */
  double kappa;         /* curvature -div n */
} node_t;

/* Faces: 0 west, 1 east, 2 south, 3 north. */
static const double face_m[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

static int face_node(const geo_t *g, int f, int k) {
  int p = g->p;
  switch (f) {
    case 0: return 0 + g->P1 * k;
    case 1: return p + g->P1 * k;
    case 2: return k;
    default: return k + g->P1 * p;
  }
}

/* Neighbour across face f, or -1 at a wall. */
static int neighbour(const geo_t *g, int e, int f) {
  int ex = e % g->nx, ey = e / g->nx;
  const int *bc = g->pr->bc;
  switch (f) {
    case 0:
      if (ex > 0) return e - 1;
      return bc[0] == ORC_BC_PERIODIC ? e + g->nx - 1 : -1;
    case 1:
      if (ex < g->nx - 1) return e + 1;
      return bc[1] == ORC_BC_PERIODIC ? e - g->nx + 1 : -1;
    case 2:
      if (ey > 0) return e - g->nx;
      return bc[2] == ORC_BC_PERIODIC ? e + g->nx * (g->ny - 1) : -1;
    default:
      if (ey < g->ny - 1) return e + g->nx;
      return bc[3] == ORC_BC_PERIODIC ? e - g->nx * (g->ny - 1) : -1;
  }
}

/* BR1 lifting of the face jumps of the nodal field f into the gradient (gx, gy):
   at every face node a of element e, M_a^-1 int_face l_a ({f} - f-) m, i.e.
   w_f / (w_a J) (f+ - f-) / 2 times the outward normal m, with f+ the
   neighbour's value at the coincident node (the own value at a wall, where
   nothing is added). */
static void lift_jumps(const geo_t *g, const double *f, double *gx, double *gy) {
  const int nf = g->dim == 2 ? 4 : 2, nk = g->dim == 2 ? g->P1 : 1;
  for (int e = 0; e < g->E; ++e)
    for (int fc = 0; fc < nf; ++fc) {
      int e2 = neighbour(g, e, fc);
      if (e2 < 0) continue;
      const double *m = face_m[fc];
      double Jf = g->dim == 2 ? 0.5 * (fc < 2 ? g->hy : g->hx) : 1.0;
      for (int k = 0; k < nk; ++k) {
        int a = face_node(g, fc, k);
        long nm = (long)e * g->Np + a, np_ = (long)e2 * g->Np + face_node(g, fc ^ 1, k);
        double wf = (g->dim == 2 ? g->wt[k] : 1.0) * Jf;
        double lift = wf / (node_weight(g, a) * g->J) * 0.5 * (f[np_] - f[nm]);
        gx[nm] += lift * m[0];
        if (gy) gy[nm] += lift * m[1];
      }
    }
}

int orc_gradients(const orc_problem *pr, const double *f, double *gx, double *gy) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < g.Np; ++a) {
      double s0 = 0.0, s1 = 0.0;
      for (int b = 0; b < g.Np; ++b) {
        double gr[2];
        grad_basis(&g, b, a, gr);
        s0 += f[(long)e * g.Np + b] * gr[0];
        s1 += f[(long)e * g.Np + b] * gr[1];
      }
      gx[(long)e * g.Np + a] = s0;
      gy[(long)e * g.Np + a] = s1;
    }
  if (pr->grad_lift) lift_jumps(&g, f, gx, gy);
  return 0;
}

/* Accumulate a contribution to R and its magnitude to the rounding scale. */
typedef struct {
  double *R, *A, *part; /* part may be NULL */
  long N;
} acc_t;

static void add(acc_t *ac, int v, long n, double val, double mag) {
  ac->R[v * ac->N + n] += val;
  ac->A[v * ac->N + n] += fabs(mag);
  if (ac->part) ac->part[v * ac->N + n] += val;
}

/* ------------------------------------------------------------------------ */
/* Right-hand side                                                          */
/* ------------------------------------------------------------------------ */

int orc_rhs(const orc_problem *pr, const double *w, double *L, double *S, double *parts) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  const long N = g.N;
  const int Np = g.Np, P1 = g.P1;
  const double Gam = pr->Gamma, eps = pr->eps;
  const double drho0 = pr->rho0[0] - pr->rho0[1];

  node_t *nd = (node_t *)calloc((size_t)N, sizeof(node_t));
  double *R = (double *)calloc((size_t)NV * N, sizeof(double));
  double *A = (double *)calloc((size_t)NV * N, sizeof(double));
  if (!nd || !R || !A) {
    free(nd); free(R); free(A);
    return -2;
  }
  if (parts) memset(parts, 0, sizeof(double) * 3 * NV * N);
  acc_t vol = {R, A, parts ? parts : NULL, N};
  acc_t srf = {R, A, parts ? parts + NV * N : NULL, N};
  acc_t src = {R, A, parts ? parts + 2 * NV * N : NULL, N};

  /* 1. Pointwise closure at every node. */
  OMP_FOR
  for (long n = 0; n < N; ++n) {
    double wn[NV];
    for (int v = 0; v < NV; ++v) wn[v] = w[v * N + n];
    closure(&g, wn, &nd[n].q);
  }

  /* 2. Broken (element-local) gradients: grad f(x_a) = sum_b f_b grad l_b(x_a). */
  OMP_FOR
  for (int e = 0; e < g.E; ++e) {
    for (int a = 0; a < Np; ++a) {
      node_t *t = &nd[(long)e * Np + a];
      for (int d = 0; d < 2; ++d) t->gphi[d] = t->gpsi[d] = t->gu[d] = t->gv[d] = 0.0;
      for (int b = 0; b < Np; ++b) {
        const node_t *s = &nd[(long)e * Np + b];
        double gr[2];
        grad_basis(&g, b, a, gr);
        for (int d = 0; d < 2; ++d) {
          t->gphi[d] += s->q.phi * gr[d];
          t->gpsi[d] += s->q.psi * gr[d];
          t->gu[d] += s->q.u * gr[d];
          t->gv[d] += s->q.v * gr[d];
        }
      }
    }
  }

  /* 2b. Broken gradients kept for the transport term; with grad_lift, the
         gradients of phi and psi become BR1-lifted (central traces). */
  for (long n = 0; n < N; ++n)
    for (int d = 0; d < 2; ++d) {
      nd[n].bphi[d] = nd[n].gphi[d];
      nd[n].bpsi[d] = nd[n].gpsi[d];
    }
  if (pr->grad_lift) {
    double *f = (double *)malloc(sizeof(double) * N), *gx = (double *)malloc(sizeof(double) * N),
           *gy = (double *)malloc(sizeof(double) * N);
    if (!f || !gx || !gy) {
      free(f); free(gx); free(gy); free(nd); free(R); free(A);
      return -2;
    }
    for (int fld = 0; fld < 2; ++fld) {
      for (long n = 0; n < N; ++n) {
        f[n] = fld == 0 ? nd[n].q.phi : nd[n].q.psi;
        gx[n] = gy[n] = 0.0;
      }
      lift_jumps(&g, f, gx, gy);
      for (long n = 0; n < N; ++n) {
        double *gr = fld == 0 ? nd[n].gphi : nd[n].gpsi;
        gr[0] += gx[n];
        gr[1] += gy[n];
      }
    }
    free(f); free(gx); free(gy);
  }

  /* 3. Normal from the level set, a_1, viscous stress. */
  OMP_FOR
  for (long n = 0; n < N; ++n) {
    node_t *t = &nd[n];
    double norm = sqrt(t->gpsi[0] * t->gpsi[0] + t->gpsi[1] * t->gpsi[1]);
    for (int d = 0; d < 2; ++d) t->n[d] = norm < 1e-12 ? 0.0 : t->gpsi[d] / norm;
    double s = t->q.phi * (1.0 - t->q.phi);
    for (int d = 0; d < 2; ++d) {
      t->a1[d] = Gam * (eps * t->gphi[d] - s * t->n[d]);
      t->a1m[d] = Gam * (fabs(eps * t->gphi[d]) + fabs(s * t->n[d]));
    }
    if (pr->viscous) {
      /* tau = 2 mu (S - (div u)/3 I), S = (grad u + grad u^T)/2 */
      double div = t->gu[0] + t->gv[1];
      double mu = t->q.mu;
      t->tau[0][0] = 2.0 * mu * (t->gu[0] - div / 3.0);
      t->tau[1][1] = 2.0 * mu * (t->gv[1] - div / 3.0);
      t->tau[0][1] = t->tau[1][0] = mu * (t->gu[1] + t->gv[0]);
    }
  }

  /* 4. Curvature kappa = -div n (broken derivative of the nodal normal). */
  if (pr->surface_tension) {
    OMP_FOR
    for (int e = 0; e < g.E; ++e)
      for (int a = 0; a < Np; ++a) {
        double div = 0.0;
        for (int b = 0; b < Np; ++b) {
          double gr[2];
          grad_basis(&g, b, a, gr);
          const node_t *s = &nd[(long)e * Np + b];
          div += s->n[0] * gr[0] + s->n[1] * gr[1];
        }
        nd[(long)e * Np + a].kappa = -div;
      }
  }

  /* 5. Volume term  sum_k w_k J grad l_a(x_k) . F_k  for the conservative
        fluxes F (moved to the right-hand side), written per equation as in
        the weak forms of Sec. 3. */
  OMP_FOR
  for (int e = 0; e < g.E; ++e) {
    for (int k = 0; k < Np; ++k) {
      const node_t *t = &nd[(long)e * Np + k];
      const prim_t *q = &t->q;
      double F[NV][2], Fm[NV][2];
      double um[2] = {fabs(q->u), fabs(q->v)};
      double vel[2] = {q->u, q->v};
      for (int d = 0; d < 2; ++d) {
        /* phi: grad . a_1 on the right  ->  flux -a_1 */
        F[ORC_PHI][d] = -t->a1[d];
        Fm[ORC_PHI][d] = t->a1m[d];
        F[ORC_PSI][d] = 0.0;
        Fm[ORC_PSI][d] = 0.0;
        /* m_l: m_l u - R_l,  R_1 = rho_1^(0) a_1,  R_2 = rho_2^(0) a_2 = -rho_2^(0) a_1 */
        F[ORC_M1][d] = q->m1 * vel[d] - pr->rho0[0] * t->a1[d];
        Fm[ORC_M1][d] = fabs(q->m1) * um[d] + pr->rho0[0] * t->a1m[d];
        F[ORC_M2][d] = q->m2 * vel[d] + pr->rho0[1] * t->a1[d];
        Fm[ORC_M2][d] = fabs(q->m2) * um[d] + pr->rho0[1] * t->a1m[d];
        /* rho u_i: rho u_i u_d + P delta_id - f_d u_i - tau_id,  f = (rho_1^0 - rho_2^0) a_1 */
        F[ORC_RU][d] = q->ru * vel[d] + (d == 0 ? q->P : 0.0) - drho0 * t->a1[d] * q->u;
        Fm[ORC_RU][d] = fabs(q->ru) * um[d] + (d == 0 ? fabs(q->P) : 0.0) + fabs(drho0) * t->a1m[d] * um[0];
        F[ORC_RV][d] = q->rv * vel[d] + (d == 1 ? q->P : 0.0) - drho0 * t->a1[d] * q->v;
        Fm[ORC_RV][d] = fabs(q->rv) * um[d] + (d == 1 ? fabs(q->P) : 0.0) + fabs(drho0) * t->a1m[d] * um[1];
        /* rho E: (rho E + P) u_d - f_d k - sum_l rho_l H_l a_l,d - (tau u)_d */
        F[ORC_RE][d] = (q->rE + q->P) * vel[d] - drho0 * t->a1[d] * q->k - q->B * t->a1[d];
        Fm[ORC_RE][d] = (fabs(q->rE) + fabs(q->P)) * um[d] + fabs(drho0) * t->a1m[d] * q->k +
                        fabs(q->B) * t->a1m[d];
        if (pr->viscous) {
          F[ORC_RU][d] -= t->tau[0][d];
          Fm[ORC_RU][d] += fabs(t->tau[0][d]);
          F[ORC_RV][d] -= t->tau[1][d];
          Fm[ORC_RV][d] += fabs(t->tau[1][d]);
          double tu = t->tau[0][d] * q->u + t->tau[1][d] * q->v;
          F[ORC_RE][d] -= tu;
          Fm[ORC_RE][d] += fabs(t->tau[0][d] * q->u) + fabs(t->tau[1][d] * q->v);
        }
      }
      double wk = node_weight(&g, k) * g.J;
      for (int a = 0; a < Np; ++a) {
        double gr[2];
        grad_basis(&g, a, k, gr);
        if (gr[0] == 0.0 && gr[1] == 0.0) continue;
        long n = (long)e * Np + a;
        for (int v = 0; v < NV; ++v) {
          double val = wk * (gr[0] * F[v][0] + gr[1] * F[v][1]);
          double mag = wk * (fabs(gr[0]) * Fm[v][0] + fabs(gr[1]) * Fm[v][1]);
          if (v == ORC_PSI) continue;
          add(&vol, v, n, val, mag);
        }
      }
    }
  }

  /* 6. Non-conservative transport -int l_a u.grad(phi) (and psi), and the
        sources of Sec. 2 (gravity, CSF surface tension). */
  OMP_FOR
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < Np; ++a) {
      long n = (long)e * Np + a;
      const node_t *t = &nd[n];
      const prim_t *q = &t->q;
      double wa = node_weight(&g, a) * g.J;
      double tphi = q->u * t->bphi[0] + q->v * t->bphi[1];
      double tpsi = q->u * t->bpsi[0] + q->v * t->bpsi[1];
      add(&vol, ORC_PHI, n, -wa * tphi, wa * (fabs(q->u * t->bphi[0]) + fabs(q->v * t->bphi[1])));
      add(&vol, ORC_PSI, n, -wa * tpsi, wa * (fabs(q->u * t->bpsi[0]) + fabs(q->v * t->bpsi[1])));
      if (pr->gravity) {
        add(&src, ORC_RU, n, wa * q->rho * pr->g[0], wa * q->rho * pr->g[0]);
        add(&src, ORC_RV, n, wa * q->rho * pr->g[1], wa * q->rho * pr->g[1]);
        double gu = q->rho * (pr->g[0] * q->u + pr->g[1] * q->v);
        add(&src, ORC_RE, n, wa * gu, wa * (fabs(q->rho * pr->g[0] * q->u) + fabs(q->rho * pr->g[1] * q->v)));
      }
      if (pr->surface_tension) {
        double dG = sqrt(t->gphi[0] * t->gphi[0] + t->gphi[1] * t->gphi[1]);
        double s = pr->sigma * t->kappa * dG;
        add(&src, ORC_RU, n, wa * s * t->n[0], wa * s * t->n[0]);
        add(&src, ORC_RV, n, wa * s * t->n[1], wa * s * t->n[1]);
        add(&src, ORC_RE, n, wa * s * (q->u * t->n[0] + q->v * t->n[1]),
            wa * (fabs(s * q->u * t->n[0]) + fabs(s * q->v * t->n[1])));
      }
    }

  /* 7. Faces.  For element e, face f and face node k: "-" = own trace,
        "+" = neighbour trace (or wall ghost), m = outward unit normal. */
  const int nf = g.dim == 2 ? 4 : 2;
  const int nk = g.dim == 2 ? P1 : 1;
  OMP_FOR
  for (int e = 0; e < g.E; ++e) {
    for (int f = 0; f < nf; ++f) {
      int e2 = neighbour(&g, e, f);
      int f2 = f ^ 1; /* opposite face of the neighbour */
      const double *m = face_m[f];
      double hperp = f < 2 ? g.hx : g.hy;
      double eta = pr->c_ip * (double)P1 * (double)P1 / hperp;
      double Jf = g.dim == 2 ? 0.5 * (f < 2 ? g.hy : g.hx) : 1.0;
      for (int k = 0; k < nk; ++k) {
        int a = face_node(&g, f, k);
        long nm = (long)e * Np + a;
        const node_t *tm = &nd[nm];
        node_t ghost;
        const node_t *tp;
        int wall = e2 < 0;
        if (!wall) {
          tp = &nd[(long)e2 * Np + face_node(&g, f2, k)];
        } else {
          ghost = *tm;
          int slip = pr->bc[f] == ORC_BC_SLIP;
          if (pr->bc[f] == ORC_BC_PRESSURE) {
            /* exterior state at rest at p_bc: rho e = P (sum phi_l g_l) + sum phi_l C_l */
            double ph1 = tm->q.phi, ph2 = 1.0 - tm->q.phi;
            double wn[NV] = {tm->q.phi, tm->q.psi, tm->q.m1, tm->q.m2, 0.0, 0.0,
                             pr->p_bc[f] * (ph1 * g.gi[0] + ph2 * g.gi[1]) + (ph1 * g.C[0] + ph2 * g.C[1])};
            closure(&g, wn, &ghost.q);
          } else if (slip) {
            double un = tm->q.ru * m[0] + tm->q.rv * m[1];
            ghost.q.ru = tm->q.ru - 2.0 * un * m[0];
            ghost.q.rv = tm->q.rv - 2.0 * un * m[1];
            double vn = tm->q.u * m[0] + tm->q.v * m[1];
            ghost.q.u = tm->q.u - 2.0 * vn * m[0];
            ghost.q.v = tm->q.v - 2.0 * vn * m[1];
          } else {
            ghost.q.ru = -tm->q.ru;
            ghost.q.rv = -tm->q.rv;
            ghost.q.u = -tm->q.u;
            ghost.q.v = -tm->q.v;
          }
          tp = &ghost;
        }
        const prim_t *qm = &tm->q, *qp = &tp->q;
        double wf = (g.dim == 2 ? g.wt[k] : 1.0) * Jf;

        double unm = qm->u * m[0] + qm->v * m[1];
        double unp = qp->u * m[0] + qp->v * m[1];
        double lam = fmax(fabs(unm) + qm->c, fabs(unp) + qp->c);

        /* Lax-Friedrichs: F.m = {F_conv}.m - lambda [[w]]  (conservative equations) */
        double Wm[NV] = {qm->phi, qm->psi, qm->m1, qm->m2, qm->ru, qm->rv, qm->rE};
        double Wp[NV] = {qp->phi, qp->psi, qp->m1, qp->m2, qp->ru, qp->rv, qp->rE};
        double Fcm[NV], Fcp[NV];
        Fcm[ORC_M1] = qm->m1 * unm;  Fcp[ORC_M1] = qp->m1 * unp;
        Fcm[ORC_M2] = qm->m2 * unm;  Fcp[ORC_M2] = qp->m2 * unp;
        Fcm[ORC_RU] = qm->ru * unm + qm->P * m[0];  Fcp[ORC_RU] = qp->ru * unp + qp->P * m[0];
        Fcm[ORC_RV] = qm->rv * unm + qm->P * m[1];  Fcp[ORC_RV] = qp->rv * unp + qp->P * m[1];
        Fcm[ORC_RE] = (qm->rE + qm->P) * unm;  Fcp[ORC_RE] = (qp->rE + qp->P) * unp;
        for (int v = ORC_M1; v <= ORC_RE; ++v) {
          double hj = 0.5 * (Wp[v] - Wm[v]);
          double Fh = 0.5 * (Fcp[v] + Fcm[v]) - lam * hj;
          double mag = 0.5 * (fabs(Fcp[v]) + fabs(Fcm[v])) + fabs(lam * hj);
          if (v == ORC_RU || v == ORC_RV) mag += fabs(qm->P) + fabs(qp->P);
          if (v == ORC_RE) mag += 0.5 * (fabs(qm->P * unm) + fabs(qp->P * unp));
          add(&srf, v, nm, -wf * Fh, wf * mag);
        }

        /* Transport of phi and psi: -m.u~phi~ + m.u^phi^ on the left-hand
           side, i.e. (lambda - m.u-) [[phi]] on the right-hand side. */
        for (int v = ORC_PHI; v <= ORC_PSI; ++v) {
          double hj = 0.5 * (Wp[v] - Wm[v]);
          add(&srf, v, nm, wf * (lam - unm) * hj, wf * (fabs(lam * hj) + fabs(unm * hj)));
        }

        /* Symmetric interior penalty flux for a_1 and every a_1-derived term. */
        if (!wall) {
          double jump = qp->phi - qm->phi;
          double gn = 0.5 * ((tp->gphi[0] + tm->gphi[0]) * m[0] + (tp->gphi[1] + tm->gphi[1]) * m[1]);
          double sp = qp->phi * (1.0 - qp->phi), sm = qm->phi * (1.0 - qm->phi);
          double sharp = 0.5 * (sp * (tp->n[0] * m[0] + tp->n[1] * m[1]) + sm * (tm->n[0] * m[0] + tm->n[1] * m[1]));
          double ahat = Gam * (eps * (gn + eta * jump) - sharp);
          double amag = Gam * (eps * (0.5 * (fabs(tp->gphi[0] * m[0] + tp->gphi[1] * m[1]) +
                                             fabs(tm->gphi[0] * m[0] + tm->gphi[1] * m[1])) +
                                      fabs(eta * jump)) +
                               0.5 * (fabs(sp) + fabs(sm)));
          double Cq[NV], Cm[NV];
          Cq[ORC_PHI] = 1.0;
          Cq[ORC_PSI] = 0.0;
          Cq[ORC_M1] = pr->rho0[0];
          Cq[ORC_M2] = -pr->rho0[1];
          Cq[ORC_RU] = drho0 * 0.5 * (qp->u + qm->u);
          Cq[ORC_RV] = drho0 * 0.5 * (qp->v + qm->v);
          Cq[ORC_RE] = 0.5 * (qp->B + qm->B) + drho0 * 0.5 * (qp->k + qm->k);
          for (int v = 0; v < NV; ++v) Cm[v] = fabs(Cq[v]);
          Cm[ORC_RU] = fabs(drho0) * 0.5 * (fabs(qp->u) + fabs(qm->u));
          Cm[ORC_RV] = fabs(drho0) * 0.5 * (fabs(qp->v) + fabs(qm->v));
          Cm[ORC_RE] = 0.5 * (fabs(qp->B) + fabs(qm->B)) + fabs(drho0) * 0.5 * (qp->k + qm->k);
          for (int v = 0; v < NV; ++v) {
            if (v == ORC_PSI) continue;
            add(&srf, v, nm, wf * Cq[v] * ahat, wf * Cm[v] * amag);
          }
          /* Symmetric term of the SIP bilinear form, lifted into the element:
             - int 1/2 Gamma eps (phi+ - phi-) grad l_b . m  for every node b. */
          double sym = 0.5 * Gam * eps * jump;
          for (int b = 0; b < Np; ++b) {
            double gr[2];
            grad_basis(&g, b, a, gr);
            double gm = gr[0] * m[0] + gr[1] * m[1];
            if (gm == 0.0) continue;
            long nb = (long)e * Np + b;
            for (int v = 0; v < NV; ++v) {
              if (v == ORC_PSI) continue;
              add(&srf, v, nb, -wf * Cq[v] * sym * gm, wf * Cm[v] * sym * gm);
            }
          }
        }

        /* Viscous interior-penalty flux. */
        if (pr->viscous) {
          double mu_avg = 0.5 * (qp->mu + qm->mu);
          double tm_m[2], tp_m[2];
          for (int d = 0; d < 2; ++d) {
            tm_m[d] = tm->tau[d][0] * m[0] + tm->tau[d][1] * m[1];
            tp_m[d] = tp->tau[d][0] * m[0] + tp->tau[d][1] * m[1];
          }
          double th_x = 0.5 * (tp_m[0] + tm_m[0]) + eta * mu_avg * (qp->u - qm->u);
          double th_y = 0.5 * (tp_m[1] + tm_m[1]) + eta * mu_avg * (qp->v - qm->v);
          add(&srf, ORC_RU, nm, wf * th_x,
              wf * (0.5 * (fabs(tp_m[0]) + fabs(tm_m[0])) + fabs(eta * mu_avg * (qp->u - qm->u))));
          add(&srf, ORC_RV, nm, wf * th_y,
              wf * (0.5 * (fabs(tp_m[1]) + fabs(tm_m[1])) + fabs(eta * mu_avg * (qp->v - qm->v))));
          double tu_m = tm_m[0] * qm->u + tm_m[1] * qm->v;
          double tu_p = tp_m[0] * qp->u + tp_m[1] * qp->v;
          double eh = 0.5 * (tu_p + tu_m) + eta * mu_avg * (qp->k - qm->k);
          add(&srf, ORC_RE, nm, wf * eh,
              wf * (0.5 * (fabs(tu_p) + fabs(tu_m)) + fabs(eta * mu_avg * (qp->k - qm->k))));
        }
      }
    }
  }

  /* 8. Apply the inverse of the diagonal (collocated) mass matrix. */
  OMP_FOR
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < Np; ++a) {
      long n = (long)e * Np + a;
      double Minv = 1.0 / (node_weight(&g, a) * g.J);
      for (int v = 0; v < NV; ++v) {
        L[v * N + n] = R[v * N + n] * Minv;
        if (S) S[v * N + n] = A[v * N + n] * Minv;
        if (parts)
          for (int s = 0; s < 3; ++s) parts[s * NV * N + v * N + n] *= Minv;
      }
    }
  free(nd);
  free(R);
  free(A);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Time stepping and diagnostics                                            */
/* ------------------------------------------------------------------------ */

int orc_rk3(const orc_problem *pr, double *w, double dt, int nsteps) {
  long N = orc_num_nodes(pr);
  if (N < 0 || nsteps < 0) return -1;
  size_t len = (size_t)NV * N;
  double *L = (double *)malloc(len * sizeof(double));
  double *w1 = (double *)malloc(len * sizeof(double));
  double *w2 = (double *)malloc(len * sizeof(double));
  if (!L || !w1 || !w2) {
    free(L); free(w1); free(w2);
    return -2;
  }
  int rc = 0;
  for (int s = 0; s < nsteps && rc == 0; ++s) {
    /* Shu-Osher form of the three-stage, third-order SSP Runge-Kutta method. */
    rc = orc_rhs(pr, w, L, NULL, NULL);
    for (size_t i = 0; i < len; ++i) w1[i] = w[i] + dt * L[i];
    if (rc == 0) rc = orc_rhs(pr, w1, L, NULL, NULL);
    for (size_t i = 0; i < len; ++i) w2[i] = 0.75 * w[i] + 0.25 * (w1[i] + dt * L[i]);
    if (rc == 0) rc = orc_rhs(pr, w2, L, NULL, NULL);
    for (size_t i = 0; i < len; ++i) w[i] = w[i] / 3.0 + 2.0 / 3.0 * (w2[i] + dt * L[i]);
  }
  free(L);
  free(w1);
  free(w2);
  return rc;
}

int orc_diag(const orc_problem *pr, const double *w, double *out) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  for (int i = 0; i < 16; ++i) out[i] = 0.0;
  out[7] = out[9] = out[11] = out[13] = INFINITY;
  out[8] = out[10] = out[12] = out[14] = -INFINITY;
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < g.Np; ++a) {
      long n = (long)e * g.Np + a;
      double wJ = node_weight(&g, a) * g.J;
      double wn[NV];
      for (int v = 0; v < NV; ++v) {
        wn[v] = w[v * g.N + n];
        out[v] += wJ * wn[v];
        if (!isfinite(wn[v])) out[15] += 1.0;
      }
      prim_t q;
      closure(&g, wn, &q);
      out[7] = fmin(out[7], q.phi);
      out[8] = fmax(out[8], q.phi);
      out[9] = fmin(out[9], q.P);
      out[10] = fmax(out[10], q.P);
      out[11] = fmin(out[11], q.u);
      out[12] = fmax(out[12], q.u);
      out[13] = fmin(out[13], q.v);
      out[14] = fmax(out[14], q.v);
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Kinematic mode (Sec. 4.1)                                                */
/* ------------------------------------------------------------------------ */

void orc_velocity_at(const orc_velocity *vel, double x, double y, double t, double *u, double *v) {
  if (vel->kind == ORC_VEL_RIDER_KOTHE) {
    double X = x - vel->xc + 0.5, Y = y - vel->yc + 0.5;
    double sx = sin(M_PI * X), sy = sin(M_PI * Y), c = cos(M_PI * t / vel->T);
    *u = sx * sx * sin(2.0 * M_PI * Y) * c;
    *v = -sin(2.0 * M_PI * X) * sy * sy * c;
  } else {
    *u = vel->u0;
    *v = vel->v0;
  }
}

double orc_stream_at(const orc_velocity *vel, double x, double y, double t) {
  if (vel->kind == ORC_VEL_RIDER_KOTHE) {
    double X = x - vel->xc + 0.5, Y = y - vel->yc + 0.5;
    double sx = sin(M_PI * X), sy = sin(M_PI * Y);
    return sx * sx * sy * sy * cos(M_PI * t / vel->T) / M_PI;
  }
  return vel->u0 * y - vel->v0 * x;
}

int orc_kin_velocity(const orc_problem *pr, const orc_velocity *vel, double t, double *u, double *v) {
  geo_t g;
  if (geo_init(&g, pr) || pr->dim != 2 || !vel) return -1;
  const long N = g.N;
  const int Np = g.Np;
  double *x = (double *)malloc(sizeof(double) * N), *y = (double *)malloc(sizeof(double) * N);
  double *psi = (double *)malloc(sizeof(double) * N);
  if (!x || !y || !psi) {
    free(x); free(y); free(psi);
    return -2;
  }
  orc_nodes(pr, x, y);
  if (vel->kind != ORC_VEL_RIDER_KOTHE) {
    for (long n = 0; n < N; ++n) orc_velocity_at(vel, x[n], y[n], t, &u[n], &v[n]);
  } else {
    for (long n = 0; n < N; ++n) psi[n] = orc_stream_at(vel, x[n], y[n], t);
    for (int e = 0; e < g.E; ++e)
      for (int a = 0; a < Np; ++a) {
        double ua = 0.0, va = 0.0;
        for (int b = 0; b < Np; ++b) {
          double gr[2];
          grad_basis(&g, b, a, gr);
          ua += psi[(long)e * Np + b] * gr[1];
          va -= psi[(long)e * Np + b] * gr[0];
        }
        u[(long)e * Np + a] = ua;
        v[(long)e * Np + a] = va;
      }
  }
  free(x); free(y); free(psi);
  return 0;
}

typedef struct {
  double phi, psi, u, v;
  double gphi[2], gpsi[2], n[2], a1[2], a1m[2];
} knode_t;

int orc_kin_rhs(const orc_problem *pr, const orc_velocity *vel, double t, const double *w, double *L,
                double *S) {
  geo_t g;
  if (geo_init(&g, pr) || pr->dim != 2 || !vel) return -1;
  for (int f = 0; f < 4; ++f)
    if (pr->bc[f] != ORC_BC_PERIODIC) return -1;
  const long N = g.N;
  const int Np = g.Np, P1 = g.P1;
  const double Gam = pr->Gamma, eps = pr->eps;
  knode_t *nd = (knode_t *)calloc((size_t)N, sizeof(knode_t));
  double *R = (double *)calloc((size_t)2 * N, sizeof(double));
  double *A = (double *)calloc((size_t)2 * N, sizeof(double));
  double *vu = (double *)malloc(sizeof(double) * N), *vv = (double *)malloc(sizeof(double) * N);
  if (!nd || !R || !A || !vu || !vv || orc_kin_velocity(pr, vel, t, vu, vv)) {
    free(nd); free(R); free(A); free(vu); free(vv);
    return -2;
  }
  acc_t ac = {R, A, NULL, N};

  /* 1. Nodal values and the nodal velocity of the scheme (orc_kin_velocity). */
  for (long n = 0; n < N; ++n) {
    nd[n].phi = w[n];
    nd[n].psi = w[N + n];
    nd[n].u = vu[n];
    nd[n].v = vv[n];
  }
  free(vu);
  free(vv);
  /* 2. Broken gradients of phi and psi. */
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < Np; ++a) {
      knode_t *k = &nd[(long)e * Np + a];
      for (int b = 0; b < Np; ++b) {
        const knode_t *s = &nd[(long)e * Np + b];
        double gr[2];
        grad_basis(&g, b, a, gr);
        for (int d = 0; d < 2; ++d) {
          k->gphi[d] += s->phi * gr[d];
          k->gpsi[d] += s->psi * gr[d];
        }
      }
    }
  /* 3. Normal and a_1 = Gamma (eps grad phi - phi (1 - phi) n). */
  for (long n = 0; n < N; ++n) {
    knode_t *k = &nd[n];
    double norm = sqrt(k->gpsi[0] * k->gpsi[0] + k->gpsi[1] * k->gpsi[1]);
    double s = k->phi * (1.0 - k->phi);
    for (int d = 0; d < 2; ++d) {
      k->n[d] = norm < 1e-12 ? 0.0 : k->gpsi[d] / norm;
      k->a1[d] = Gam * (eps * k->gphi[d] - s * k->n[d]);
      k->a1m[d] = Gam * (fabs(eps * k->gphi[d]) + fabs(s * k->n[d]));
    }
  }
  /* 4. Volume terms: int grad l_a . (-a_1) for phi, and the non-conservative
        transport -int l_a u . grad f for phi and psi. */
  for (int e = 0; e < g.E; ++e)
    for (int k = 0; k < Np; ++k) {
      const knode_t *q = &nd[(long)e * Np + k];
      double wk = node_weight(&g, k) * g.J;
      for (int a = 0; a < Np; ++a) {
        double gr[2];
        grad_basis(&g, a, k, gr);
        if (gr[0] == 0.0 && gr[1] == 0.0) continue;
        long n = (long)e * Np + a;
        add(&ac, 0, n, -wk * (gr[0] * q->a1[0] + gr[1] * q->a1[1]),
            wk * (fabs(gr[0]) * q->a1m[0] + fabs(gr[1]) * q->a1m[1]));
      }
      long n = (long)e * Np + k;
      add(&ac, 0, n, -wk * (q->u * q->gphi[0] + q->v * q->gphi[1]),
          wk * (fabs(q->u * q->gphi[0]) + fabs(q->v * q->gphi[1])));
      add(&ac, 1, n, -wk * (q->u * q->gpsi[0] + q->v * q->gpsi[1]),
          wk * (fabs(q->u * q->gpsi[0]) + fabs(q->v * q->gpsi[1])));
    }
  /* 5. Faces: transport (lambda - m.u-) [[f]] with lambda = max(|u-.m|, |u+.m|),
        and the SIP flux of a_1 with its symmetric term (phi only). */
  for (int e = 0; e < g.E; ++e)
    for (int f = 0; f < 4; ++f) {
      int e2 = neighbour(&g, e, f);
      const double *m = face_m[f];
      double hperp = f < 2 ? g.hx : g.hy;
      double eta = pr->c_ip * (double)P1 * (double)P1 / hperp;
      double Jf = 0.5 * (f < 2 ? g.hy : g.hx);
      for (int k = 0; k < P1; ++k) {
        long nm = (long)e * Np + face_node(&g, f, k);
        const knode_t *tm = &nd[nm];
        const knode_t *tp = &nd[(long)e2 * Np + face_node(&g, f ^ 1, k)];
        double wf = g.wt[k] * Jf;
        double unm = tm->u * m[0] + tm->v * m[1];
        double unp = tp->u * m[0] + tp->v * m[1];
        double lam = fmax(fabs(unm), fabs(unp));
        double hj_phi = 0.5 * (tp->phi - tm->phi), hj_psi = 0.5 * (tp->psi - tm->psi);
        add(&ac, 0, nm, wf * (lam - unm) * hj_phi, wf * (fabs(lam * hj_phi) + fabs(unm * hj_phi)));
        add(&ac, 1, nm, wf * (lam - unm) * hj_psi, wf * (fabs(lam * hj_psi) + fabs(unm * hj_psi)));
        double jump = tp->phi - tm->phi;
        double gn = 0.5 * ((tp->gphi[0] + tm->gphi[0]) * m[0] + (tp->gphi[1] + tm->gphi[1]) * m[1]);
        double sp = tp->phi * (1.0 - tp->phi), sm = tm->phi * (1.0 - tm->phi);
        double sharp = 0.5 * (sp * (tp->n[0] * m[0] + tp->n[1] * m[1]) + sm * (tm->n[0] * m[0] + tm->n[1] * m[1]));
        double ahat = Gam * (eps * (gn + eta * jump) - sharp);
        double amag = Gam * (eps * (0.5 * (fabs(tp->gphi[0] * m[0] + tp->gphi[1] * m[1]) +
                                           fabs(tm->gphi[0] * m[0] + tm->gphi[1] * m[1])) +
                                    fabs(eta * jump)) +
                             0.5 * (fabs(sp) + fabs(sm)));
        add(&ac, 0, nm, wf * ahat, wf * amag);
        double sym = 0.5 * Gam * eps * jump;
        int a = face_node(&g, f, k);
        for (int b = 0; b < Np; ++b) {
          double gr[2];
          grad_basis(&g, b, a, gr);
          double gm = gr[0] * m[0] + gr[1] * m[1];
          if (gm == 0.0) continue;
          add(&ac, 0, (long)e * Np + b, -wf * sym * gm, wf * sym * gm);
        }
      }
    }
  /* 6. Inverse of the diagonal mass matrix. */
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < Np; ++a) {
      long n = (long)e * Np + a;
      double Minv = 1.0 / (node_weight(&g, a) * g.J);
      for (int v = 0; v < 2; ++v) {
        L[v * N + n] = R[v * N + n] * Minv;
        if (S) S[v * N + n] = A[v * N + n] * Minv;
      }
    }
  free(nd); free(R); free(A);
  return 0;
}

int orc_kin_rk4(const orc_problem *pr, const orc_velocity *vel, double *w, double t0, double dt, int nsteps) {
  long N = orc_num_nodes(pr);
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
  for (int s = 0; s < nsteps && rc == 0; ++s) {
    /* Classical RK4: k1 = L(w, t), k2 = L(w + dt/2 k1, t + dt/2),
       k3 = L(w + dt/2 k2, t + dt/2), k4 = L(w + dt k3, t + dt),
       w <- w + dt/6 (k1 + 2 k2 + 2 k3 + k4), summed in that order. */
    double t = t0 + s * dt;
    rc = orc_kin_rhs(pr, vel, t, w, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] = k[i]; ws[i] = w[i] + 0.5 * dt * k[i]; }
    if (rc == 0) rc = orc_kin_rhs(pr, vel, t + 0.5 * dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] += 2.0 * k[i]; ws[i] = w[i] + 0.5 * dt * k[i]; }
    if (rc == 0) rc = orc_kin_rhs(pr, vel, t + 0.5 * dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) { acc[i] += 2.0 * k[i]; ws[i] = w[i] + dt * k[i]; }
    if (rc == 0) rc = orc_kin_rhs(pr, vel, t + dt, ws, k, NULL);
    for (size_t i = 0; i < len; ++i) w[i] = w[i] + dt / 6.0 * (acc[i] + k[i]);
  }
  free(k); free(acc); free(ws);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Level-set re-initialisation (end of Sec. 3)                              */
/* ------------------------------------------------------------------------ */

/* Broken gradient of the nodal field f at every node. */
static void broken_gradient(const geo_t *g, const double *f, double *gx, double *gy) {
  for (int e = 0; e < g->E; ++e)
    for (int a = 0; a < g->Np; ++a) {
      double s0 = 0.0, s1 = 0.0;
      for (int b = 0; b < g->Np; ++b) {
        double gr[2];
        grad_basis(g, b, a, gr);
        s0 += f[(long)e * g->Np + b] * gr[0];
        s1 += f[(long)e * g->Np + b] * gr[1];
      }
      gx[(long)e * g->Np + a] = s0;
      gy[(long)e * g->Np + a] = s1;
    }
}

int orc_reinit_sign(const orc_problem *pr, const double *phi, double *S) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  const long N = g.N;
  double *p0 = (double *)malloc(sizeof(double) * N), *gx = (double *)malloc(sizeof(double) * N),
         *gy = (double *)malloc(sizeof(double) * N);
  if (!p0 || !gx || !gy) {
    free(p0); free(gx); free(gy);
    return -2;
  }
  for (long n = 0; n < N; ++n) p0[n] = phi[n] - 0.5;
  broken_gradient(&g, p0, gx, gy);
  for (long n = 0; n < N; ++n) {
    double gm = sqrt(gx[n] * gx[n] + gy[n] * gy[n]);
    if (gm < 1e-12 || !(pr->eps > 0.0)) S[n] = p0[n] > 0.0 ? 1.0 : (p0[n] < 0.0 ? -1.0 : 0.0);
    else S[n] = tanh(p0[n] / (2.0 * pr->eps * gm));
  }
  free(p0); free(gx); free(gy);
  return 0;
}

int orc_reinit_rhs(const orc_problem *pr, const double *S, const double *psi, double nu, double *L) {
  geo_t g;
  if (geo_init(&g, pr)) return -1;
  const long N = g.N;
  const int Np = g.Np, P1 = g.P1;
  double *gx = (double *)malloc(sizeof(double) * N), *gy = (double *)malloc(sizeof(double) * N);
  double *R = (double *)calloc((size_t)N, sizeof(double));
  if (!gx || !gy || !R) {
    free(gx); free(gy); free(R);
    return -2;
  }
  broken_gradient(&g, psi, gx, gy);
  /* Source S (1 - |grad psi|) (the sign that drives |grad psi| to 1, see the
     header) and volume term int grad l_a . (-nu grad psi). */
  for (int e = 0; e < g.E; ++e)
    for (int k = 0; k < Np; ++k) {
      long nk = (long)e * Np + k;
      double wk = node_weight(&g, k) * g.J;
      double gm = sqrt(gx[nk] * gx[nk] + gy[nk] * gy[nk]);
      R[nk] += wk * S[nk] * (1.0 - gm);
      for (int a = 0; a < Np; ++a) {
        double gr[2];
        grad_basis(&g, a, k, gr);
        R[(long)e * Np + a] += -wk * nu * (gr[0] * gx[nk] + gr[1] * gy[nk]);
      }
    }
  /* Faces: SIP flux nu ({grad psi}.m + eta (psi+ - psi-)) and the symmetric
     term -1/2 nu (psi+ - psi-) grad l_b . m; nothing through walls. */
  const int nf = g.dim == 2 ? 4 : 2, nk = g.dim == 2 ? P1 : 1;
  for (int e = 0; e < g.E; ++e)
    for (int f = 0; f < nf; ++f) {
      int e2 = neighbour(&g, e, f);
      if (e2 < 0) continue;
      const double *m = face_m[f];
      double hperp = f < 2 ? g.hx : g.hy;
      double eta = pr->c_ip * (double)P1 * (double)P1 / hperp;
      double Jf = g.dim == 2 ? 0.5 * (f < 2 ? g.hy : g.hx) : 1.0;
      for (int k = 0; k < nk; ++k) {
        int a = face_node(&g, f, k);
        long nm = (long)e * Np + a, np_ = (long)e2 * Np + face_node(&g, f ^ 1, k);
        double wf = (g.dim == 2 ? g.wt[k] : 1.0) * Jf;
        double jump = psi[np_] - psi[nm];
        double gn = 0.5 * ((gx[np_] + gx[nm]) * m[0] + (gy[np_] + gy[nm]) * m[1]);
        R[nm] += wf * nu * (gn + eta * jump);
        for (int b = 0; b < Np; ++b) {
          double gr[2];
          grad_basis(&g, b, a, gr);
          double gmb = gr[0] * m[0] + gr[1] * m[1];
          if (gmb != 0.0) R[(long)e * Np + b] += -wf * 0.5 * nu * jump * gmb;
        }
      }
    }
  for (int e = 0; e < g.E; ++e)
    for (int a = 0; a < Np; ++a) {
      long n = (long)e * Np + a;
      L[n] = R[n] / (node_weight(&g, a) * g.J);
    }
  free(gx); free(gy); free(R);
  return 0;
}

int orc_reinit(const orc_problem *pr, const double *phi, double *psi, int niter, double nu, double dtau) {
  long N = orc_num_nodes(pr);
  if (N < 0 || niter < 0) return -1;
  double *S = (double *)malloc(sizeof(double) * N), *L = (double *)malloc(sizeof(double) * N);
  double *p1 = (double *)malloc(sizeof(double) * N), *p2 = (double *)malloc(sizeof(double) * N);
  if (!S || !L || !p1 || !p2) {
    free(S); free(L); free(p1); free(p2);
    return -2;
  }
  int rc = orc_reinit_sign(pr, phi, S);
  for (long n = 0; n < N; ++n) psi[n] = phi[n] - 0.5;
  for (int it = 0; it < niter && rc == 0; ++it) {
    rc = orc_reinit_rhs(pr, S, psi, nu, L);
    for (long n = 0; n < N; ++n) p1[n] = psi[n] + dtau * L[n];
    if (rc == 0) rc = orc_reinit_rhs(pr, S, p1, nu, L);
    for (long n = 0; n < N; ++n) p2[n] = 0.75 * psi[n] + 0.25 * (p1[n] + dtau * L[n]);
    if (rc == 0) rc = orc_reinit_rhs(pr, S, p2, nu, L);
    for (long n = 0; n < N; ++n) psi[n] = psi[n] / 3.0 + 2.0 / 3.0 * (p2[n] + dtau * L[n]);
  }
  free(S); free(L); free(p1); free(p2);
  return rc;
}

