// dg_kin.cuh -- kinematic mode (Sec. 4.1): the phase field and the level set
// advected by a prescribed analytical velocity, FP64 (GB300, sm_103a).
//
//   d(phi)/dt + u . grad(phi) = div a_1,   a_1 = Gamma (eps grad phi - phi (1 - phi) n),
//   d(psi)/dt + u . grad(psi) = 0,         n = grad psi / |grad psi|,
//
// with the discretisation of the phi and psi rows of the full scheme: the
// weak-form volume term of -a_1 (sum-factorised Dhat contractions), the
// non-conservative transport -u . grad f at the nodes, the transport flux
// (lambda - m.u-) [[f]] with lambda = max(|u-.m|, |u+.m|) -- the advection
// speed alone, as the kinematic system has no sound speed -- and the SIP flux
// of a_1 with its lifted symmetric term.  The velocity is the analytical field
// sampled at each node.  Time integration is the classical four-stage
// Runge-Kutta method, fused into the surface kernel.  Periodic meshes only.
#pragma once

#include <math_constants.h>

#include "dg_common.cuh"
#include "dg_kernels_fp64.cuh"

namespace dgpf {

enum { VEL_UNIFORM = 0, VEL_RIDER_KOTHE = 1 };
// What the kinematic surface kernel writes: the right-hand side, or one stage
// of classical RK4 (w0: step start, acc: k1 + 2 k2 + 2 k3 so far).
enum KinMode { KIN_RHS = 0, KIN_K1 = 1, KIN_K2 = 2, KIN_K3 = 3, KIN_K4 = 4 };
// Kinematic face-trace record: phi, psi, d(phi)/d(axis), n_axis, u_axis.
enum { K_PHI = 0, K_PSI, K_GPHI, K_N, K_U, NT_KIN };

// Constants of one triangle type of the split-rectangle mesh (dg_tri.cuh): det = d(x,y)/d(r,s),
// its inverse, the inverse-map derivatives, and per edge f the outward unit normal m, half the
// edge length, the penalty eta_tri / h_e and the reference components of grad l . m
// (gr = rx m0 + ry m1, gs = sx m0 + sy m1).
struct TriConst {
  double det, idet, rx, ry, sx, sy;
  double m0[3], m1[3], hl[3], eta[3], gr[3], gs[3];
};

struct KinParams {
  int nx, ny, E, N;
  double x0, y0, hx, hy;
  double Gamma, eps, eta_x, eta_y;
  int vel;                 // VEL_UNIFORM or VEL_RIDER_KOTHE
  double u0, v0, T;        // uniform velocity; Rider-Kothe period
  double xc, yc;           // Rider-Kothe vortex centre
  double eta_tri;          // triangles: c_ip (p+1)(p+2); the edge penalty is eta_tri / h_e
  TriConst tc[2];          // triangles: the two element types
  const double *vel_tab;   // spatial velocity factor U at every node (rectangles) or quadrature point
                           // (triangles), see kin_velocity_factor
  const double *ops;       // operator table (OpsLayout)
  const double *xi;        // GLL nodes on [-1, 1]
  const double *t0;        // device: time at the start of the captured step sequence
  int check_finite;
  unsigned *status;
};

// Prescribed velocity (Sec. 4.1), u(x, t) = c(t) U(x): the Rider-Kothe vortex with
// c = cos(pi t / T) and U = (sin^2(pi X) sin(2 pi Y), -sin(2 pi X) sin^2(pi Y)), or c = 1 and
// U = (u0, v0).  U does not change between stages: it is evaluated once per node (rectangles) or
// quadrature point (triangles) when the context is created, into KinParams::vel_tab, and a stage
// multiplies by c -- the FP64 sines would otherwise cost more than the scheme.
__device__ __forceinline__ void kin_velocity_factor(const KinParams &kp, double x, double y, double *U,
                                                    double *V) {
  if (kp.vel == VEL_RIDER_KOTHE) {
    const double X = x - kp.xc + 0.5, Y = y - kp.yc + 0.5;
    const double sx = sin(CUDART_PI * X), sy = sin(CUDART_PI * Y);
    *U = sx * sx * sin(2.0 * CUDART_PI * Y);
    *V = -sin(2.0 * CUDART_PI * X) * sy * sy;
  } else {
    *U = kp.u0;
    *V = kp.v0;
  }
}

__device__ __forceinline__ double kin_time_factor(const KinParams &kp, double t) {
  return kp.vel == VEL_RIDER_KOTHE ? cos(CUDART_PI * t / kp.T) : 1.0;
}

// U at every node of the rectangles, [N][2].
template <int P>
__global__ void k_kin_velocity_table(const KinParams kp, double *__restrict__ tab) {
  constexpr int P1 = P + 1, NP = P1 * P1;
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const int e = (int)(n / NP), a = (int)(n % NP), i = a % P1, j = a / P1;
  const int ex = e % kp.nx, ey = e / kp.nx;
  const double x = kp.x0 + kp.hx * (ex + 0.5 * (__ldg(kp.xi + i) + 1.0));
  const double y = kp.y0 + kp.hy * (ey + 0.5 * (__ldg(kp.xi + j) + 1.0));
  kin_velocity_factor(kp, x, y, &tab[2 * n], &tab[2 * n + 1]);
}

template <int P>
cudaError_t launch_kin_velocity_table(const KinParams &kp, double *tab, cudaStream_t s) {
  k_kin_velocity_table<P><<<(unsigned)((kp.N + 255) / 256), 256, 0, s>>>(kp, tab);
  return cudaGetLastError();
}

// Volume kernel: broken gradients, n, a_1, the volume term of -a_1, the
// non-conservative transport of phi and psi, and the face traces.  The stage
// time is *kp.t0 + (step dt) + (stage offset), as the two host-side parts
// tstep = step index x dt and toff = stage fraction x dt.
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_kin_volume(const KinParams kp, double tstep, double toff, const double *__restrict__ w, double *__restrict__ rvol,
             double *__restrict__ tr) {
  using G = Geom<P, 2, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int P11 = P1 * P1;
  __shared__ double s_op[4 * P11];
  __shared__ double s_f[2][EPB][NP];
  for (int t = threadIdx.x; t < 4 * P11; t += blockDim.x) s_op[t] = kp.ops[t];
  const double *Dx = s_op, *Dy = s_op + P11, *Dhx = s_op + 2 * P11, *Dhy = s_op + 3 * P11;

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < kp.E;
  const int i = a % P1, j = a / P1;
  const int N = kp.N;
  const long n = (long)(act ? e : 0) * NP + a;

  const double phi = act ? __ldg(w + n) : 0.0, psi = act ? __ldg(w + N + n) : 0.0;
  const double c = kin_time_factor(kp, (*kp.t0 + tstep) + toff);
  const double2 U = __ldg(reinterpret_cast<const double2 *>(kp.vel_tab) + n);
  const double u = U.x * c, v = U.y * c;

  if (lane) {
    s_f[0][le][a] = phi;
    s_f[1][le][a] = psi;
  }
  __syncthreads();
  double gpx = 0.0, gpy = 0.0, gsx = 0.0, gsy = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const double dx = Dx[i * P1 + c], dy = Dy[j * P1 + c];
    gpx = fma(dx, s_f[0][le][c + P1 * j], gpx);
    gsx = fma(dx, s_f[1][le][c + P1 * j], gsx);
    gpy = fma(dy, s_f[0][le][i + P1 * c], gpy);
    gsy = fma(dy, s_f[1][le][i + P1 * c], gsy);
  }
  const double g2 = gsx * gsx + gsy * gsy;
  double nx = 0.0, ny = 0.0;
  if (g2 >= 1e-24) {
    const double r = rsqrt(g2);
    nx = gsx * r;
    ny = gsy * r;
  }
  const double sphi = phi * (1.0 - phi);
  const double a1x = kp.Gamma * (kp.eps * gpx - sphi * nx);
  const double a1y = kp.Gamma * (kp.eps * gpy - sphi * ny);
  __syncthreads();
  if (lane) {
    s_f[0][le][a] = -a1x;
    s_f[1][le][a] = -a1y;
  }
  __syncthreads();
  double Rphi = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    Rphi = fma(Dhx[i * P1 + c], s_f[0][le][c + P1 * j], Rphi);
    Rphi = fma(Dhy[j * P1 + c], s_f[1][le][i + P1 * c], Rphi);
  }
  Rphi -= u * gpx + v * gpy;
  const double Rpsi = -(u * gsx + v * gsy);
  if (act) {
    rvol[n] = Rphi;
    rvol[N + n] = Rpsi;
  }
  const bool onW = i == 0, onE = i == P, onS = j == 0, onN = j == P;
  if (act && (onW || onE || onS || onN)) {
    const long base = (long)e * NFK, stride = (long)kp.E * NFK;
    auto put = [&](int f, int kk, double gn, double nn, double ua) {
      const long o = base + f * NK + kk;
      tr[K_PHI * stride + o] = phi;
      tr[K_PSI * stride + o] = psi;
      tr[K_GPHI * stride + o] = gn;
      tr[K_N * stride + o] = nn;
      tr[K_U * stride + o] = ua;
    };
    if (onW) put(0, j, gpx, nx, u);
    if (onE) put(1, j, gpx, nx, u);
    if (onS) put(2, i, gpy, ny, v);
    if (onN) put(3, i, gpy, ny, v);
  }
}

// Periodic neighbour across face f (0 W, 1 E, 2 S, 3 N).
__device__ __forceinline__ int kin_neighbour(const KinParams &kp, int e, int f) {
  const int ex = e % kp.nx, ey = e / kp.nx;
  switch (f) {
    case 0: return ex > 0 ? e - 1 : e + kp.nx - 1;
    case 1: return ex < kp.nx - 1 ? e + 1 : e - kp.nx + 1;
    case 2: return ey > 0 ? e - kp.nx : e + kp.nx * (kp.ny - 1);
    default: return ey < kp.ny - 1 ? e + kp.nx : e - kp.nx * (kp.ny - 1);
  }
}

// Surface kernel: transport and SIP fluxes at the face nodes, lifting of the
// symmetric term, M^-1, and the right-hand side or an RK4 stage:
//   K1: acc = L,        out = w0 + dt/2 L
//   K2: acc += 2 L,     out = w0 + dt/2 L
//   K3: acc += 2 L,     out = w0 + dt L
//   K4: out = w0 + dt/6 (acc + L)   (out may be w0: each node is read, then
//                                    written, by the same thread)
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_kin_surface(const KinParams kp, int mode, double dt, const double *w0, const double *__restrict__ rvol,
              const double *__restrict__ tr, double *__restrict__ acc, double *out) {
  using G = Geom<P, 2, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  const OpsLayout L{P1, NP};
  __shared__ double s_op[4 * P1 * P1 + 3 * P1 + NP];
  __shared__ double s_surf[EPB][NFK][2];
  __shared__ double s_lift[EPB][NFK];
  for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = kp.ops[t];
  __syncthreads();
  const double *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy();
  const double *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < kp.E;
  const long stride = (long)kp.E * NFK;

  for (int t = a; t < NFK && lane; t += NP) {
    const int f = t / NK, kk = t % NK;
    const bool xf = f < 2;
    const double sg = (f & 1) ? 1.0 : -1.0;
    double Tm[NT_KIN], Tp[NT_KIN];
    if (act) {
      const int e2 = kin_neighbour(kp, e, f);
      const long om = (long)e * NFK + t, op = (long)e2 * NFK + (f ^ 1) * NK + kk;
#pragma unroll
      for (int q = 0; q < NT_KIN; ++q) {
        Tm[q] = __ldg(tr + q * stride + om);
        Tp[q] = __ldg(tr + q * stride + op);
      }
    } else {
#pragma unroll
      for (int q = 0; q < NT_KIN; ++q) Tm[q] = Tp[q] = 0.0;
    }
    const double unm = Tm[K_U] * sg, unp = Tp[K_U] * sg;
    const double lam = fmax(fabs(unm), fabs(unp));
    const double wf = xf ? wfx[kk] : wfy[kk];
    const double eta = xf ? kp.eta_x : kp.eta_y;
    const double jump = Tp[K_PHI] - Tm[K_PHI];
    const double gn = 0.5 * (Tp[K_GPHI] + Tm[K_GPHI]) * sg;
    const double sharp =
        0.5 * (Tp[K_PHI] * (1.0 - Tp[K_PHI]) * Tp[K_N] + Tm[K_PHI] * (1.0 - Tm[K_PHI]) * Tm[K_N]) * sg;
    const double ahat = kp.Gamma * (kp.eps * (gn + eta * jump) - sharp);
    s_surf[le][t][0] = wf * (lam - unm) * 0.5 * jump + wf * ahat;
    s_surf[le][t][1] = wf * (lam - unm) * 0.5 * (Tp[K_PSI] - Tm[K_PSI]);
    s_lift[le][t] = -wf * 0.5 * kp.Gamma * kp.eps * jump;
  }
  __syncthreads();
  if (!act) return;

  const int i = a % P1, j = a / P1;
  double sp = 0.0, ss = 0.0;
  if (i == 0) { sp += s_surf[le][0 * NK + j][0]; ss += s_surf[le][0 * NK + j][1]; }
  if (i == P) { sp += s_surf[le][1 * NK + j][0]; ss += s_surf[le][1 * NK + j][1]; }
  if (j == 0) { sp += s_surf[le][2 * NK + i][0]; ss += s_surf[le][2 * NK + i][1]; }
  if (j == P) { sp += s_surf[le][3 * NK + i][0]; ss += s_surf[le][3 * NK + i][1]; }
  sp += s_lift[le][0 * NK + j] * -Dx[0 * P1 + i] + s_lift[le][1 * NK + j] * Dx[P * P1 + i];
  sp += s_lift[le][2 * NK + i] * -Dy[0 * P1 + j] + s_lift[le][3 * NK + i] * Dy[P * P1 + j];
  const double im = invM[a];
  const long n = (long)e * NP + a;
  const int N = kp.N;
  const double Lv[2] = {__ldg(rvol + n) + sp * im, __ldg(rvol + N + n) + ss * im};
  bool bad = false;
#pragma unroll
  for (int vv = 0; vv < 2; ++vv) {
    const long o = (long)vv * N + n;
    double r;
    if (mode == KIN_RHS) {
      r = Lv[vv];
    } else {
      const double base = w0[o];
      if (mode == KIN_K1) {
        acc[o] = Lv[vv];
        r = base + 0.5 * dt * Lv[vv];
      } else if (mode == KIN_K2) {
        acc[o] += 2.0 * Lv[vv];
        r = base + 0.5 * dt * Lv[vv];
      } else if (mode == KIN_K3) {
        acc[o] += 2.0 * Lv[vv];
        r = base + dt * Lv[vv];
      } else {
        r = base + dt / 6.0 * (acc[o] + Lv[vv]);
      }
    }
    bad |= !isfinite(r);
    out[o] = r;
  }
  if (kp.check_finite && bad) atomicOr(kp.status, STATUS_NONFINITE);
}

struct KinKernels {
  cudaError_t (*volume)(const KinParams &, double tstep, double toff, const double *w, double *rvol, double *tr,
                        cudaStream_t);
  cudaError_t (*velocity_table)(const KinParams &, double *tab, cudaStream_t);
  cudaError_t (*surface)(const KinParams &, int mode, double dt, const double *w0, const double *rvol,
                         const double *tr, double *acc, double *out, cudaStream_t);
};

template <int P>
cudaError_t launch_kin_volume(const KinParams &kp, double tstep, double toff, const double *w, double *rvol,
                              double *tr, cudaStream_t s) {
  using G = Geom<P, 2, false, false>;
  k_kin_volume<P><<<(kp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(kp, tstep, toff, w, rvol, tr);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_kin_surface(const KinParams &kp, int mode, double dt, const double *w0, const double *rvol,
                               const double *tr, double *acc, double *out, cudaStream_t s) {
  using G = Geom<P, 2, false, false>;
  k_kin_surface<P><<<(kp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(kp, mode, dt, w0, rvol, tr, acc, out);
  return cudaGetLastError();
}

bool kin_kernels(int p, KinKernels *out);

}  // namespace dgpf
