/*
 * dg_oracle.h -- plain FP64 CPU oracle for the DG right-hand side of the
 * quasi-conservative five-equation two-phase model coupled to the Allen-Cahn
 * phase field and an advected level set (Tonicello & Ihme, arXiv 2306.05002).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU library
 * against the paper.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * State layout (shared with the library only as a documented convention):
 *   w[v * N + e * Np + a],  v = 0..6 = [phi, psi, m1, m2, rho_u, rho_v, rho_E]
 *   N  = E * Np,  E = nx * ny elements, e = ex + nx * ey,
 *   Np = (p+1)^dim,  a = i + (p+1) * j with (i, j) the GLL node indices.
 *   phi = phi_1 (volume fraction of phase 1), m_l = rho_l phi_l.
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NV 7
enum { ORC_PHI = 0, ORC_PSI = 1, ORC_M1 = 2, ORC_M2 = 3, ORC_RU = 4, ORC_RV = 5, ORC_RE = 6 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_NOSLIP = 1, ORC_BC_SLIP = 2, ORC_BC_PRESSURE = 3 };

typedef struct {
  int dim;            /* 1 or 2 */
  int nx, ny;         /* elements per direction (ny = 1 when dim = 1) */
  int p;              /* polynomial order, 1..8 */
  double x0, x1, y0, y1;
  int bc[4];          /* west, east, south, north */
  double gamma[2], pinf[2], rho0[2], mu[2];   /* phase 1, phase 2 */
  double sigma;       /* surface tension coefficient */
  double g[2];        /* gravitational acceleration */
  double Gamma, eps;  /* Allen-Cahn velocity scale and interface thickness */
  double c_ip;        /* interior-penalty constant: eta = c_ip (p+1)^2 / h */
  int viscous, gravity, surface_tension;
  double p_bc[4];     /* exterior pressure of ORC_BC_PRESSURE sides */
  int grad_lift;      /* 1: BR1-lifted gradients of phi and psi (see orc_gradients) */
} orc_problem;

/* GLL nodes xi[0..p] (ascending) and weights wt[0..p] on [-1, 1]. */
int orc_gll(int p, double *xi, double *wt);
/* D[a*(p+1)+b] = l_b'(xi_a), derivative of the b-th Lagrange polynomial. */
int orc_lagrange_deriv(int p, const double *xi, double *D);
/* Total number of nodes E * Np. */
long orc_num_nodes(const orc_problem *pr);
/* Physical coordinates of every node (y may be NULL for dim = 1). */
int orc_nodes(const orc_problem *pr, double *x, double *y);
/* Primitive variables at every node: prim[q * N + n], q = rho, u, v, P, c, B. */
int orc_primitives(const orc_problem *pr, const double *w, double *prim);
/*
 * Gradient of the nodal field f (N values) at every node: the broken
 * (element-local) gradient, plus, when pr->grad_lift is set, the BR1 lifting of
 * the face jumps: q = grad_h f + M^-1 sum over faces of int l (f^ - f-) m with
 * the central trace f^ = {f} (at walls and pressure boundaries the exterior
 * value is the own, so nothing is lifted there).
 */
int orc_gradients(const orc_problem *pr, const double *f, double *gx, double *gy);
/*
 * L = M^-1 R(w).  S (nullable) receives the sum of absolute values of every
 * contribution to R, also scaled by M^-1, which sets the rounding scale for
 * parity checks.  parts (nullable, 3 * 7 * N) receives the volume (including
 * the non-conservative transport), surface (including the symmetric interior
 * penalty term) and source parts of L separately.
 */
int orc_rhs(const orc_problem *pr, const double *w, double *L, double *S, double *parts);

/* Threads of the OpenMP build (liboracle_omp.so): n > 0 sets the count; returns
   the count in use (1 in the plain build). */
int orc_threads(int n);

/* nsteps of three-stage SSP Runge-Kutta (Shu-Osher form), in place. */
int orc_rk3(const orc_problem *pr, double *w, double dt, int nsteps);
/*
 * Kinematic mode (Sec. 4.1, "kinematic tests"): only the phase field and the
 * level set, advected by a prescribed analytical velocity u(x, t):
 *   d(phi)/dt + u . grad(phi) = div a_1,   d(psi)/dt + u . grad(psi) = 0,
 * with a_1 as in the full model.  State w[v * N + n], v = 0 (phi), 1 (psi).
 * Velocity kinds: uniform (u0, v0); Rider-Kothe vortex with period T about
 * the centre (xc, yc), with X = x - xc + 1/2, Y = y - yc + 1/2:
 *   u = sin^2(pi X) sin(2 pi Y) cos(pi t / T),
 *   v = -sin(2 pi X) sin^2(pi Y) cos(pi t / T)
 * (xc = yc = 1/2 is the formula as printed in Sec. 4.1).
 * Periodic boundaries only.
 */
#define ORC_KIN_NV 2
enum { ORC_VEL_UNIFORM = 0, ORC_VEL_RIDER_KOTHE = 1 };
typedef struct {
  int kind;
  double u0, v0;   /* uniform velocity */
  double T;        /* Rider-Kothe period */
  double xc, yc;   /* Rider-Kothe vortex centre: the printed formula is xc = yc = 1/2 */
} orc_velocity;

/* Velocity at (x, y) and time t. */
void orc_velocity_at(const orc_velocity *vel, double x, double y, double t, double *u, double *v);
/* Stream function Psi at (x, y) and time t: u = dPsi/dy, v = -dPsi/dx
   (Rider-Kothe: sin^2(pi X) sin^2(pi Y) cos(pi t / T) / pi; uniform: u0 y - v0 x). */
double orc_stream_at(const orc_velocity *vel, double x, double y, double t);
/* The nodal velocity of the kinematic scheme at time t (u, v: N values each): a uniform field as
   given; the Rider-Kothe vortex as the discrete curl of its stream function interpolated at each
   element's nodes, (dPsi_h/dy, -dPsi_h/dx) with the element's derivative matrices, so that its
   discrete divergence vanishes and its normal component is continuous across faces. */
int orc_kin_velocity(const orc_problem *pr, const orc_velocity *vel, double t, double *u, double *v);
/* L = M^-1 R(w) of the kinematic system at time t; S (nullable) as in orc_rhs. */
int orc_kin_rhs(const orc_problem *pr, const orc_velocity *vel, double t, const double *w, double *L,
                double *S);
/* nsteps of the classical four-stage Runge-Kutta method from time t0, in place. */
int orc_kin_rk4(const orc_problem *pr, const orc_velocity *vel, double *w, double t0, double dt, int nsteps);

/*
 * Kinematic mode on triangles (the paper's mesh (b)): each Cartesian cell of
 * the periodic rectangle split along its rising diagonal into two
 * counter-clockwise triangles (element 2 (i + nx j) + type, type 0 = lower
 * right, 1 = upper left), nodal basis of degree p <= 4 on equispaced nodes,
 * collapsed Gauss-Legendre volume rule of (p+2)^2 points, (p+2)-point edge
 * rule, full element mass matrix; see dg_oracle_tri.c.  State (2, N) with
 * N = 2 nx ny (p+1)(p+2)/2.  Uses dim, nx, ny, p, domain, Gamma, eps, c_ip.
 */
long orc_tri_num_nodes(const orc_problem *pr);
int orc_tri_nodes(const orc_problem *pr, double *x, double *y);
int orc_tri_integral(const orc_problem *pr, const double *f, double *out);
int orc_tri_mass(const orc_problem *pr, int e, double *M);
int orc_tri_rhs(const orc_problem *pr, const orc_velocity *vel, double t, const double *w, double *L, double *S);
int orc_tri_rk4(const orc_problem *pr, const orc_velocity *vel, double *w, double t0, double dt, int nsteps);

/*
 * Level-set re-initialisation (end of Sec. 3): the pseudo-time equation
 *   d(psi)/d(tau) = S (1 - |grad psi|) + div(nu grad psi),   psi(0) = psi0 = phi - 1/2,
 * (the sign under which |grad psi| relaxes to 1; the paper prints the
 * hyperbolic term with the opposite sign on the left-hand side)
 * with the smeared sign S = tanh(psi0 / (2 eps |grad psi0|)) fixed from psi0.
 * The hyperbolic term is a nodal source (broken gradient); the diffusion uses
 * the SIP flux nu ({grad psi}.m + eta (psi+ - psi-)) with its symmetric term and
 * no flux through walls; pseudo-time integration is three-stage SSP RK.
 */
/* S at every node from psi0 = phi - 1/2. */
int orc_reinit_sign(const orc_problem *pr, const double *phi, double *S);
/* L = M^-1 R(psi) of the re-initialisation equation for the sign S. */
int orc_reinit_rhs(const orc_problem *pr, const double *S, const double *psi, double nu, double *L);
/* psi <- psi0 = phi - 1/2, then niter SSP-RK3 steps of size dtau. */
int orc_reinit(const orc_problem *pr, const double *phi, double *psi, int niter, double nu, double dtau);

/*
 * Diagnostics: out[0..6] = integrals of the 7 variables, out[7..8] = min/max
 * phi, out[9..10] = min/max P, out[11..12] = min/max u, out[13..14] =
 * min/max v, out[15] = number of non-finite state entries.
 */
int orc_diag(const orc_problem *pr, const double *w, double *out16);

#ifdef __cplusplus
}
#endif
#endif
