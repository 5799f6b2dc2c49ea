// dg_common.cuh -- definitions shared by the kernels and the host side of
// libdgpf (GB300, sm_103a).  Tonicello & Ihme, arXiv 2306.05002.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dgpf {

constexpr int NV = 7;
// State variables, Sec. 2: phase field, level set, partial densities,
// momentum, total energy.
enum Var { PHI = 0, PSI = 1, M1 = 2, M2 = 3, RU = 4, RV = 5, RE = 6 };
// What the surface kernel writes: the right-hand side itself, or one stage
// of the three-stage SSP Runge-Kutta method in Shu-Osher form.
enum Mode { MODE_RHS = 0, MODE_S1 = 1, MODE_S2 = 2, MODE_S3 = 3 };
enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_SLIP = 2, BC_PRESSURE = 3 };

// Face-trace record written by the volume kernel for every face node
// (element-major, one record per (element, face, node along the face)).
enum TraceField {
  T_PHI = 0, T_PSI, T_M1, T_M2, T_RU, T_RV, T_RE,  // the seven state values
  T_U, T_V, T_P, T_C, T_B,                          // velocity, pressure, mixture sound speed, B
  T_GPHI,                                           // d(phi)/d(axis normal to the face)
  T_N,                                              // level-set normal component on that axis
  T_TX, T_TY, T_MU                                  // viscous: tau . e_axis and mixture mu
};
constexpr int NT_INVISCID = 14;
constexpr int NT_VISCOUS = 17;

constexpr unsigned STATUS_NONFINITE = 1u;
constexpr unsigned STATUS_NONPHYSICAL = 2u;
constexpr unsigned STATUS_BOUNDS = 4u;  // bounds-checked build: an index left its array

// Index check of the bounds-checked build (compiled with -DDG_CHECK), the
// stand-in for a memory checker: i in [0, n) passes; a failed check latches
// STATUS_BOUNDS in the status word (when there is one) and the caller skips
// the access.  In the normal build it is the constant true.
__device__ __forceinline__ bool in_bounds(unsigned *status, long long i, long long n) {
#ifdef DG_CHECK
  if (i >= 0 && i < n) return true;
  if (status) atomicOr(status, STATUS_BOUNDS);
  return false;
#else
  (void)status;
  (void)i;
  (void)n;
  return true;
#endif
}

// Everything the kernels need about one problem, passed by value.
struct Params {
  int nx, ny, E, N;          // elements per direction, elements, nodes
  int bc[4];                 // west, east, south, north
  double p_bc[4];            // exterior pressure of BC_PRESSURE sides
  // stiffened-gas closure (Sec. 2): C_l = gamma_l Pinf_l/(gamma_l-1), g_l = 1/(gamma_l-1),
  // B = rho_1 H_1 - rho_2 H_2 = P * Bp + dC
  double C1, C2, g1, g2, Bp, dC;
  double rho01, rho02, drho0;  // reference densities rho_l^(0) and their difference
  double mu1, mu2, sigma, gx, gy;
  double Gamma, eps;
  double eta_x, eta_y;       // interior penalty on faces normal to x and to y
  int gravity, check_finite;
  int grad_lift;             // BR1-lifted gradients of phi and psi (dg_opts.grad_lift)
  const double *ops;         // operator tables, see OpsLayout
  unsigned *status;          // latched device status bits
  const double *dt_dev;      // step size read at run time (captured step sequences), else NULL
};

// Layout of the per-context operator table (device memory, doubles):
//   Dx  [P1*P1]  (2/hx) D,   D[a][b] = l_b'(xi_a)
//   Dy  [P1*P1]  (2/hy) D
//   Dhx [P1*P1]  (2/hx) Dhat, Dhat[i][c] = w_c D[c][i] / w_i  (weak-form derivative)
//   Dhy [P1*P1]  (2/hy) Dhat
//   wt  [P1]     GLL weights
//   invM[Np]     1 / (w_i w_j J)  (inverse of the collocated mass matrix)
//   wfx [P1]     w_k * J_f on faces normal to x (1D: 1)
//   wfy [P1]     w_k * J_f on faces normal to y
struct OpsLayout {
  int P1, Np;
  __host__ __device__ int Dx() const { return 0; }
  __host__ __device__ int Dy() const { return P1 * P1; }
  __host__ __device__ int Dhx() const { return 2 * P1 * P1; }
  __host__ __device__ int Dhy() const { return 3 * P1 * P1; }
  __host__ __device__ int wt() const { return 4 * P1 * P1; }
  __host__ __device__ int invM() const { return 4 * P1 * P1 + P1; }
  __host__ __device__ int wfx() const { return 4 * P1 * P1 + P1 + Np; }
  __host__ __device__ int wfy() const { return 4 * P1 * P1 + 2 * P1 + Np; }
  __host__ __device__ int size() const { return 4 * P1 * P1 + 3 * P1 + Np; }
};

// Launch interface of one kernel family (one order, dimension and term set).
struct KernelSet {
  cudaError_t (*volume)(const Params &, const double *w, double *rvol, double *trace, cudaStream_t);
  cudaError_t (*surface)(const Params &, int mode, double dt, const double *w0, const double *ws,
                         const double *rvol, const double *trace, double *out, cudaStream_t);
  int nt;       // trace fields per face node
  int epb;      // elements per block
  int threads;  // threads per block
};

// Kernel families by order (defined in dg_inst_p<P>.cu).
bool kernels_fp64(int p, int dim, bool viscous, bool surface_tension, KernelSet *out);

}  // namespace dgpf
