/*
 * dgpf.h -- C ABI of libdgpf, a GB300 (sm_103a) implementation of the explicit
 * Discontinuous Galerkin right-hand side of Tonicello & Ihme, "A high-order
 * diffused-interface approach for two-phase compressible flow simulations
 * using a Discontinuous Galerkin framework" (arXiv 2306.05002), driving a
 * three-stage SSP Runge-Kutta step.
 *
 * The equations are the system of Sec. 2 (phase field phi = phi_1, level set
 * psi, partial densities m_l = rho_l phi_l, momentum rho u, total energy rho E,
 * interface flux a_1 = Gamma (eps grad phi - phi (1 - phi) n) with
 * n = grad psi/|grad psi|, stiffened-gas closure, optional viscous stress,
 * gravity and CSF surface tension), discretised as in Sec. 3: nodal DG on
 * Cartesian quadrilaterals (or 1D segments) with the Lagrange basis on
 * Gauss-Lobatto-Legendre nodes and collocated quadrature, Lax-Friedrichs
 * fluxes for the conservative equations, the quasi-conservative transport
 * fluxes of Sec. 3 for phi and psi, and the symmetric interior penalty flux
 * for every a_1-derived term.
 *
 * Conventions (all entry points):
 *   - State layout: one contiguous array of 7 * N doubles, variable-major:
 *       w[v * N + e * Np + a],  v = phi, psi, m1, m2, rho u, rho v, rho E,
 *       N = E * Np nodes, E = nx * ny elements, e = ex + nx * ey,
 *       Np = (p+1)^dim, a = i + (p+1) j with (i, j) the GLL node indices.
 *     In 1D the rho v slot exists and stays zero.
 *   - Pointers named w, L, lam are DEVICE pointers unless stated otherwise;
 *     the caller owns them.  The library owns its operator tables and
 *     workspace, allocated in dg_create and freed in dg_destroy; rhs and step
 *     calls allocate nothing.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.  Launch-time
 *     errors are returned; conditions the GPU detects (non-finite values)
 *     are latched in a device status word and reported by dg_status_read.
 *     The FP32-bulk kernels of a grid that fits on the GPU at once run as
 *     programmatic dependent launches and let the kernel after them on the
 *     stream be scheduled early: a caller's kernel launched with
 *     programmatic stream serialization must call
 *     cudaGridDependencySynchronize() before it reads their results, as
 *     CUDA requires of any such launch.  Ordinary launches, copies and
 *     events on the stream are ordered as usual.
 *   - A context is not thread-safe.  No C++ exception crosses this boundary.
 *   - Failure returns a negative dg_status; dg_last_error gives a message.
 */
#ifndef DGPF_H
#define DGPF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,          /* invalid argument (message in dg_last_error) */
  DG_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  DG_ERR_OOM = -3,          /* device allocation failed */
  DG_ERR_TIMEOUT = -4,      /* a bounded device wait expired */
  DG_ERR_NONFINITE = -5,    /* the device saw a non-finite value */
  DG_ERR_NONPHYSICAL = -6,  /* the device saw rho <= 0 or P + Pinf <= 0 */
  DG_ERR_UNSUPPORTED = -7,  /* valid request the library does not implement */
  DG_ERR_BOUNDS = -8        /* bounds-checked build only: a kernel index left its array */
} dg_status;

enum { DG_BC_PERIODIC = 0, DG_BC_NOSLIP = 1, DG_BC_SLIP = 2, DG_BC_PRESSURE = 3 };
enum { DG_FP64 = 0, DG_FP32_BULK = 1 };

/* Cartesian mesh of nx * ny elements on [x0,x1] x [y0,y1] (dim = 2) or nx
   segments on [x0,x1] (dim = 1, ny must be 1).  bc = west, east, south, north;
   periodic sides must be paired.  The paper's element partition (Sec. 3).
   Boundaries (Sec. 4.2): DG_BC_NOSLIP and DG_BC_SLIP walls (ghost state = own
   state with the velocity, or its normal component, reversed), and
   DG_BC_PRESSURE, the Riemann-invariant boundary "with zero velocity and
   constant pressure" of the Rayleigh-Taylor and rising-bubble tests: the
   exterior state of the boundary Riemann problem is the own phase field,
   level set and partial densities at rest at pressure p_bc[side], and the
   Lax-Friedrichs flux between the two carries it in.  No a_1 flux crosses a
   wall or a pressure boundary, and ghost gradients equal the own ones.
   p_bc is read for DG_BC_PRESSURE sides only.
   elem: DG_ELEM_QUAD (0, the default of a zeroed struct) for the nx x ny
   rectangles (the paper's mesh (a)); DG_ELEM_TRI (1) splits every rectangle
   along its rising diagonal into two triangles, the paper's mesh (b), Sec. 4.1
   -- the kinematic mode only (dg_kin_create); the full-model calls reject it
   with DG_ERR_UNSUPPORTED. */
typedef struct {
  int dim;
  int nx, ny;
  double x0, x1, y0, y1;
  int bc[4];
  double p_bc[4];
  int elem;
} dg_mesh;

enum { DG_ELEM_QUAD = 0, DG_ELEM_TRI = 1 };

/* Phase constants of the stiffened-gas closure (Sec. 2): gamma_l, Pinf_l, the
   reference densities rho_l^(0) of R_l = rho_l^(0) a_l, viscosities mu_l
   (mixture mu = mu_1 phi + mu_2 (1 - phi)), surface tension sigma and gravity
   g.  Index 0 is phase 1 (the phase whose volume fraction is phi). */
typedef struct {
  double gamma[2], pinf[2], rho0[2], mu[2];
  double sigma;
  double g[2];
} dg_eos;

/* Options.  prec: DG_FP64 or DG_FP32_BULK.  c_ip: interior-penalty constant,
   eta = c_ip (p+1)^2 / h (<= 0 selects 1).  viscous, gravity,
   surface_tension: enable those terms of Sec. 2.  check_finite: latch
   DG_ERR_NONFINITE when an output is not finite, and DG_ERR_NONPHYSICAL when
   a state the kernels read has rho <= 0, a mixture 1/(gamma - 1) <= 0 or
   P + Pinf_mix <= 0 (the stiffened-gas closure of Sec. 2 has no real sound
   speed there).  The state is never clipped.  batch_tile (batches
   only): 0 lets the first dg_batch_step tune the tile of every order; 1..4
   fixes tile variant batch_tile - 1 for all orders (see dg_batch_step);
   other values are DG_ERR_ARG.  grad_lift: 0 (the default) takes the
   gradients of phi and psi element by element (broken gradients); 1 takes
   them BR1-lifted, the broken gradient plus M^-1 times the face integrals of
   l ({f} - f-) m (central traces; nothing is lifted at walls and pressure
   boundaries), for a_1, the level-set normal, the SIP flux's {grad phi} and
   the CSF delta -- the non-conservative transport keeps the broken gradient.
   Sec. 3 leaves the gradient discretisation open.  The lifted gradients are
   built by the FP64 kernels: FP32-bulk and batch contexts reject grad_lift = 1
   with DG_ERR_UNSUPPORTED, and such a context has no discrete adjoint. */
typedef struct {
  int prec;
  double c_ip;
  int viscous, gravity, surface_tension;
  int check_finite;
  int batch_tile;
  int grad_lift;
} dg_opts;

typedef struct dg_ctx dg_ctx;

/* Create a solver for one mesh, order p (1..5 in 2D, 1..5 in 1D), closure,
   Allen-Cahn velocity scale Gamma >= 0 and thickness eps >= 0 (Sec. 2).
   opts may be NULL (FP64, c_ip = 1, no viscous/gravity/surface terms).
   Allocates all device memory the context will use on the current device
   (except the staging buffer of dg_step_host, allocated on its first staged
   call, and the device copy of a page-locked host state, allocated on the
   first FP32-bulk single step of one).
   On success *out receives the context; on failure *out is NULL. */
dg_status dg_create(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                    const dg_opts *opts, dg_ctx **out);

/* Free the context and its device memory (NULL is ignored).  Synchronises
   the device first. */
void dg_destroy(dg_ctx *ctx);

/* Number of doubles of one state array: 7 * E * (p+1)^dim. */
size_t dg_state_len(const dg_ctx *ctx);

/* L = M^-1 R(w): the semi-discrete right-hand side of the weak form of Sec. 3
   (eq. "weakDG") for all seven equations.  w and L are device arrays of
   dg_state_len doubles and must not overlap. */
dg_status dg_rhs(dg_ctx *ctx, const double *w, double *L, void *stream);

/* Advance w (device, in place) by nsteps steps of the three-stage SSP
   Runge-Kutta method (Shu-Osher form) with step dt > 0.  nsteps = 0 is a
   no-op.  The step sequence is captured once in a CUDA graph per state array
   w and replayed; the context keeps the graphs of the two state arrays used
   most recently (a caller alternating two buffers captures once per buffer),
   and the first call for any other w pays a capture.  The graphs
   read the step size from device memory (set on stream when dt changes), so a
   caller that varies dt from call to call pays no capture for it. */
dg_status dg_step(dg_ctx *ctx, double *w, double dt, int nsteps, void *stream);

/* dg_step on a HOST state w_host (dg_state_len doubles); returns when
   w_host holds the state after nsteps SSP-RK3 steps.  FP32-bulk contexts
   with a page-locked, device-mapped w_host (cudaHostAlloc / cudaHostRegister
   memory, e.g. a pinned torch tensor) read and write it in place from the
   kernels over the host link: the first stage reads the FP64 state, the last
   stage writes it (a single step also leaves a device copy of the state it
   read, dg_state_len doubles allocated on first use and kept until
   dg_destroy, and adds its last increment to that copy, so the state
   crosses the link once each way; DG_ERR_OOM if that allocation fails).
   dg_step given such a pointer does the same.  Otherwise the state is copied to a device staging buffer
   (dg_state_len doubles, allocated on the first such call and kept until
   dg_destroy; DG_ERR_OOM if that fails), stepped and copied back, all on
   stream; pageable memory works but is staged by the driver.  No Sec. of the
   paper corresponds: this is the host-side form of dg_step. */
dg_status dg_step_host(dg_ctx *ctx, double *w_host, double dt, int nsteps, void *stream);

/* FP64 diagnostics of w (Sec. 4.1 mass error): out (HOST, 16 doubles) gets
   the integrals of the 7 variables (GLL quadrature), min/max phi, min/max P,
   min/max u, min/max v, and the count of non-finite state entries.
   Synchronises the stream. */
dg_status dg_diag(dg_ctx *ctx, const double *w, double *out, void *stream);

/* Read and clear the device status word (synchronises the stream): DG_OK,
   DG_ERR_BOUNDS (bounds-checked build only, reported first: a kernel index
   left its array), DG_ERR_NONPHYSICAL (reported before DG_ERR_NONFINITE when
   both were latched: a non-physical state is what makes the values
   non-finite) or DG_ERR_NONFINITE.  Batch contexts latch no value checks, so
   they return DG_OK or, in the bounds-checked build, DG_ERR_BOUNDS. */
dg_status dg_status_read(dg_ctx *ctx, void *stream);

/* Whether this library is the bounds-checked build (1) or the normal one (0).
   The bounds-checked build (compiled with DG_CHECK; libdgpf_check.so) checks
   the index of every global access of the library's kernels on a context
   (the two-phase model's FP64, FP32-bulk and batched kernels, the adjoint,
   kinematic, triangle and re-initialisation kernels: node, face-record,
   velocity-table and neighbour indices) against its array's extent; a failed
   check skips the access and latches a status bit, which dg_status_read
   reports as DG_ERR_BOUNDS.  failures (HOST, may be NULL) receives the number
   of such reports so far in this process, counting bits still latched when a
   context is destroyed (0 in the normal build).  dg_rhs_noalloc has no
   context to report through: its kernels check, but nothing counts them.
   The normal build compiles the checks out. */
int dg_check_build(long long *failures);

/* Self-test of the bounds-checked build: runs the FP64 volume kernel of a
   small problem with a node count one short of the mesh's (every array keeps
   its true size, so no access leaves its allocation) and returns 1 when the
   last node's index check caught it (latched and skipped), 0 when it did not,
   DG_ERR_CUDA on a CUDA failure and DG_ERR_UNSUPPORTED in the normal build.
   Synchronises stream; the planted failure is not counted by dg_check_build. */
int dg_check_selftest(void *stream);

/* Message of the last failure on this context (or of the last failed
   dg_create when ctx is NULL).  Never NULL. */
const char *dg_last_error(const dg_ctx *ctx);

/* Kernel-level timing for roofline reports: for each kernel kind, run nrep
   launches on w back to back on stream between two CUDA events and write
   the mean duration per launch in milliseconds to ms_out
   (index 0 volume kernel, 1 surface kernel, and for FP32-bulk contexts 2 the
   fused kernel that dg_step runs: the surface part of one stage followed by
   the volume part of the next, 3 the volume kernel of a call's first stage,
   which reads the FP64 state, and 4 the surface kernel of a call's last
   stage, which writes it -- into a temporary FP64 array that this call
   allocates and frees); returns the number of kinds written (<= nmax), or
   -1.  w is not modified.  Synchronises the stream. */
int dg_time_kernels(dg_ctx *ctx, const double *w, int nrep, double *ms_out, int nmax, void *stream);

/* Number of kernel launches one dg_step call of nsteps >= 0 steps makes on
   this context (the kernels of its graphs; the step-size update when dt
   changes is not counted): FP64 6 per step (a volume and a surface kernel per
   stage); FP32-bulk 1 + 3 nsteps (the first stage's volume kernel, then per
   stage one fused surface + next-volume kernel, the last stage's surface
   kernel alone).  -1 for a NULL, batch or kinematic context or nsteps < 0. */
int dg_step_launches(const dg_ctx *ctx, int nsteps);

/* Algorithmic FP64-equivalent flop and DRAM byte counts per launch of each
   kernel kind (same indexing as dg_time_kernels), from the formulas of the
   scheme (not from counters); returns the number of kinds written (<= nmax),
   or -1. */
int dg_kernel_costs(const dg_ctx *ctx, double *flops_out, double *bytes_out, int nmax);

/* Discrete adjoint of the right-hand side: out = (dL/dw)^T lam at the state
   w, the exact transpose of the Jacobian of dg_rhs (all seven equations, the
   closure, normals, a_1, fluxes and SIP lifting of Sec. 2-3 differentiated by
   hand).  Provided for FP64 contexts without viscous and surface-tension
   terms (else DG_ERR_UNSUPPORTED).  w, lam, out: device arrays of
   dg_state_len doubles; out must not overlap w or lam.  Where the two
   one-sided wave speeds of the Lax-Friedrichs lambda tie, the derivative is
   taken on the element's own side. */
dg_status dg_rhs_vjp(dg_ctx *ctx, const double *w, const double *lam, double *out, void *stream);

/* Reverse of one SSP-RK3 step: lam_n = (d w_{n+1} / d w_n)^T lam_np1 for the
   step of size dt taken from w_n (device arrays).  The two intermediate
   stages are recomputed from w_n, then three adjoint right-hand sides run in
   reverse stage order.  lam_n may alias lam_np1 (not w_n).  Same
   availability as dg_rhs_vjp.  Asynchronous on stream. */
dg_status dg_adjoint_step(dg_ctx *ctx, const double *w_n, const double *lam_np1, double *lam_n, double dt,
                          void *stream);

/* Taped step for reverse sweeps.  dg_tape_len: doubles of one step's tape
   (the two intermediate stages and the face traces of the three stages; 0 when
   the context has no adjoint).  dg_step_tape: one SSP-RK3 step of w in place
   (identical to dg_step with nsteps = 1) whose kernels write the stages and
   traces into tape (device, dg_tape_len doubles).  dg_adjoint_step_tape: the
   reverse of that step, lam_n = (d w_{n+1}/d w_n)^T lam_np1, from w_n and the
   tape, with no recomputation (three adjoint right-hand sides).  A
   checkpointed reverse sweep replays each segment with dg_step_tape and
   walks back with dg_adjoint_step_tape.  Same availability as dg_rhs_vjp. */
size_t dg_tape_len(const dg_ctx *ctx);
dg_status dg_step_tape(dg_ctx *ctx, double *w, double dt, double *tape, void *stream);
dg_status dg_adjoint_step_tape(dg_ctx *ctx, const double *w_n, const double *tape, const double *lam_np1,
                               double *lam_n, double dt, void *stream);

/* One checkpoint segment of a reverse sweep in a single call: from the
   segment's checkpoint w_start (device, dg_state_len doubles), replay m taped
   SSP-RK3 steps of size dt, keeping each step's start in states (device,
   (m + 1) * dg_state_len doubles; states[j] = w_j, states[m] = the segment's
   end) and its tape in tapes (device, m * dg_tape_len doubles), then run the m
   reverse steps, lam <- (d w_{j+1} / d w_j)^T lam from j = m - 1 down to 0, in
   place on lam (device, dg_state_len doubles).  The sequence is captured in a
   CUDA graph on the first call for a given (m, dt, states, tapes, lam) and
   replayed (the context keeps two such graphs), so a sweep's launches do not
   depend on the caller's issue rate.  Same availability as dg_rhs_vjp.
   Asynchronous on stream.  No Sec. of the paper corresponds: this is the
   checkpointed driver of the discrete adjoint. */
dg_status dg_adjoint_segment(dg_ctx *ctx, const double *w_start, int m, double dt, double *states, double *tapes,
                             double *lam, void *stream);

/* Batched ensemble: n independent 2D problems (each with its own mesh, order
   p[k] in 1..5, closure eos[k], Gamma[k], eps[k]) advanced together by the
   FP32-bulk path.  opts applies to all problems; opts->prec must be
   DG_FP32_BULK, viscous and surface_tension must be 0 (gravity is allowed).
   Problems of one order share one launch per kernel: the grid is the
   concatenation of every problem's element tiles, each block locates its
   problem through a first-block table and stages that problem's descriptor in
   shared memory.  All device memory is allocated here (one pool).
   dg_state_len of a batch context is the sum of the problems' state lengths;
   the single-problem calls reject a batch context with DG_ERR_ARG. */
dg_status dg_batch_create(int n, const dg_mesh *meshes, const int *p, const dg_eos *eos, const double *Gamma,
                          const double *eps, const dg_opts *opts, dg_ctx **out);

/* Advance every problem k of a batch by nsteps SSP-RK3 steps with its own step
   dt[k] > 0.  w (HOST array of n pointers) gives each problem's DEVICE state
   (layout as dg_step, in place); dt is a HOST array of n doubles.  The whole
   step is one CUDA graph with one branch per order (captured on the first
   call; it reads the problem descriptors from device memory, so new pointers
   or step sizes only re-upload the descriptors).  Before the capture, the
   first call tunes the tile of every order: it times NVAR = 4 compiled
   variants (elements per block: the single-problem rule or twice it;
   registers: the compiler's choice or at most 64 per thread) on the batch's
   own first-stage and fused kernels, which read the states and write only
   internal buffers, and keeps the fastest (synchronises the stream once).
   nsteps = 0 is a no-op.  Otherwise asynchronous on stream. */
dg_status dg_batch_step(dg_ctx *ctx, double *const *w, const double *dt, int nsteps, void *stream);

/* Tiles chosen by the tuner of dg_batch_step, one entry per order present
   (in order of first appearance): order p, elements per block, minimum
   resident blocks per SM asked of the compiler (1: no register cap), and the
   tuned time in ms of the stage-1 volume and two fused launches with the
   chosen and with the default tile (any output pointer may be NULL).
   Returns the number of entries written (<= nmax), 0 before the first
   dg_batch_step, -1 for a context that is not a batch. */
int dg_batch_tiles(const dg_ctx *ctx, int *p, int *epb, int *minb, double *ms_best, double *ms_default, int nmax);

/* ---------------------------------------------------------------------------
   Kinematic mode (Sec. 4.1, "kinematic tests"): the phase field phi and the
   level set psi alone, advected by a prescribed analytical velocity,
     d(phi)/dt + u . grad(phi) = div a_1,   d(psi)/dt + u . grad(psi) = 0,
   discretised as the phi and psi rows of the full scheme (the transport speed
   of the face flux is max(|u-.m|, |u+.m|): the kinematic system has no sound
   speed) and integrated with the classical four-stage Runge-Kutta method, as
   in the paper's Rider-Kothe test.  FP64.  The state is 2 x N doubles:
   w[v * N + e * Np + a], v = 0 (phi), 1 (psi), layout as dg_rhs.
   --------------------------------------------------------------------------- */
typedef enum { DG_VEL_UNIFORM = 0, DG_VEL_RIDER_KOTHE = 1 } dg_velocity_kind;

/* Prescribed velocity.  DG_VEL_UNIFORM: (u0, v0).  DG_VEL_RIDER_KOTHE: the
   vortex of Sec. 4.1 with period T > 0 about the centre (xc, yc), with
   X = x - xc + 1/2 and Y = y - yc + 1/2,
     u = sin^2(pi X) sin(2 pi Y) cos(pi t / T),
     v = -sin(2 pi X) sin^2(pi Y) cos(pi t / T)
   (xc = yc = 1/2 gives the formula as printed in Sec. 4.1). */
typedef struct {
  int kind;
  double u0, v0;
  double T;
  double xc, yc;
} dg_velocity;

/* Create a kinematic-mode context: 2D mesh with periodic boundaries on all
   four sides, order p (1..5 on rectangles, 1..4 on triangles), Allen-Cahn
   Gamma >= 0 and eps >= 0, velocity, interior-penalty constant c_ip (<= 0
   selects 1), at most 2^26 cells and fewer than 2^31 nodes per field.
   dg_state_len gives 2 N; dg_destroy releases it; the
   single-problem and batch calls of the full model reject it (DG_ERR_ARG).
   Errors as dg_create.
   Rectangles (DG_ELEM_QUAD): GLL nodes, collocated quadrature, penalty
   eta = c_ip (p+1)^2 / h.  Triangles (DG_ELEM_TRI, the paper's mesh (b)):
   triangle 2 (i + nx j) + t of cell (i, j) has the counter-clockwise vertices
   (x_i, y_j), (x_i+1, y_j), (x_i+1, y_j+1) for t = 0 and (x_i, y_j),
   (x_i+1, y_j+1), (x_i, y_j+1) for t = 1; a nodal basis of degree p on the
   (p+1)(p+2)/2 equispaced nodes of each triangle (see dg_kin_nodes), volume
   integrals by the collapsed Gauss-Legendre rule of (p+2)^2 points, edge
   integrals by (p+2)-point Gauss-Legendre, the full element mass matrix,
   penalty eta = c_ip (p+1)(p+2) / h_e with h_e = 2 |T| / |e|. */
dg_status dg_kin_create(const dg_mesh *mesh, int p, double Gamma, double eps, const dg_velocity *vel, double c_ip,
                        dg_ctx **out);

/* Node coordinates of the kinematic-mode state of mesh and order p (host
   arrays x, y of N = dg_state_len / 2 doubles each; host computation, no
   device needed).  Element-major; within a rectangle the (p+1)^2 GLL nodes
   x-fastest; within a triangle the equispaced nodes (r, s) = (-1 + 2i/p,
   -1 + 2j/p), i + j <= p, i fastest, mapped by x = v1 + (1 + r)/2 (v2 - v1) +
   (1 + s)/2 (v3 - v1).  DG_ERR_ARG / DG_ERR_UNSUPPORTED as dg_kin_create. */
dg_status dg_kin_nodes(const dg_mesh *mesh, int p, double *x, double *y);

/* L = M^-1 R(w) of the kinematic system at time t (device arrays of
   dg_state_len doubles; must not overlap). */
dg_status dg_kin_rhs(dg_ctx *ctx, const double *w, double t, double *L, void *stream);

/* Advance w (device, in place) from time t0 by nsteps classical RK4 steps of
   size dt > 0.  Captured once in a CUDA graph per state array w (the graphs
   read the start time and the step size from device memory, so t0 and dt
   may change freely).  Asynchronous on stream. */
dg_status dg_kin_step(dg_ctx *ctx, double *w, double t0, double dt, int nsteps, void *stream);

/* Level-set re-initialisation (end of Sec. 3): replace the level set psi of
   the state w (device; phi and psi are fields 0 and 1 of a full-model or a
   kinematic state; the other fields are left unchanged) by the solution after
   niter pseudo-time steps of
     d(psi)/d(tau) = S (1 - |grad psi|) + div(nu grad psi),  psi(0) = phi - 1/2,
     S = tanh(psi0 / (2 eps |grad psi0|)) (the smeared sign, fixed from psi0),
   the hyperbolic term a nodal source, the diffusion with the SIP flux and its
   symmetric term (no flux through walls), three-stage SSP Runge-Kutta of step
   dtau.  The hyperbolic term carries the sign under which |grad psi| relaxes
   to 1 (the paper prints the opposite sign, under which it grows).  nu <= 0
   selects nu = h / (2 (p + 1)) and dtau <= 0 selects
   min(0.5 h / (2p + 1), 0.1 h^2 / ((2p + 1)^2 nu)), h the smallest element
   width.  The paper applies ~50 iterations every 2000 steps.  FP64; works on
   FP64 and FP32-bulk contexts alike (on the FP64 state).  The first call
   allocates the context's re-initialisation workspace (4 N doubles and the
   face traces), kept until dg_destroy.  Rectangles only: a triangle context
   gives DG_ERR_UNSUPPORTED.  Asynchronous on stream. */
dg_status dg_reinit(dg_ctx *ctx, double *w, int niter, double nu, double dtau, void *stream);

/* Measured multiply-add rate of the current GPU in TFLOP/s (2 flops per FMA):
   kind 0 FP64, kind 1 FP32; every resident thread runs 8 independent FMA
   chains for iters rounds, timed with CUDA events on stream (synchronises
   it).  The roofline denominators of the FP64 kernels.  No Sec. of the paper
   corresponds.  DG_ERR_ARG for a bad kind, iters < 1 or a NULL output. */
dg_status dg_peak_flops(int kind, int iters, double *tflops, void *stream);

/* Size of the fixed device scratch used by dg_rhs_noalloc (32 MiB per GPU). */
#define DG_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* The FP64 right-hand side L = M^-1 R(w), as dg_rhs computes it, for callers
   that cannot allocate device memory: code that runs inside a framework's
   memory pool or under an allocator that forbids raw cudaMalloc after
   start-up, or a process that has already reserved all device memory.  The
   paper has no counterpart: this is a deployment variant of dg_rhs.
   It takes the problem description of dg_create directly (no context), plus a
   device state w and a device output L (7 * E * (p+1)^dim doubles each, not
   overlapping), and makes no device allocation and no allocating library
   call.  Its scratch (operator table, volume part, face traces) is one
   file-scope device array of DG_NOALLOC_SCRATCH_BYTES that every GPU loading
   this library holds until the process exits; a problem whose scratch would
   not fit (about 190,000 nodes at p = 3 in 2D, e.g. 64 x 64 elements fits)
   is rejected with DG_ERR_ARG before any GPU work.  Every other argument is
   checked as dg_create checks it, with the same status codes (every boundary
   kind, viscous, gravity and surface-tension terms are supported); opts->prec
   DG_FP32_BULK gives DG_ERR_UNSUPPORTED; the device status word is not
   reported.
   The first call on a device looks up the array's device address on that
   device (loading the library's module there if needed).  The operator table
   reaches the device as a kernel argument, not by a copy from host memory.
   Every call uses the same array and leaves its contents
   behind; the call writes its operator table and clears what must start at
   zero itself.  Calls whose work overlaps on the GPU (other streams, other
   host threads) race on the scratch: serialise them.  Asynchronous on
   stream. */
dg_status dg_rhs_noalloc(const dg_mesh *mesh, int p, const dg_eos *eos, double Gamma, double eps,
                         const dg_opts *opts, const double *w, double *L, void *stream);

#ifdef __cplusplus
}
#endif
#endif
