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
// of a_1 with its lifted symmetric term.  The nodal velocity is a uniform field
// as given, or, for the Rider-Kothe vortex, the discrete curl of its stream
// function interpolated at each element's nodes (discretely divergence-free,
// normal components continuous across faces: the phase field's mass is then
// conserved to round-off).  Time integration is the classical four-stage
// Runge-Kutta method; each stage is one launch (k_kin_stage), which also
// evaluates the neighbours' face traces from their nodal values.  Periodic
// meshes only.
#pragma once

#include <math_constants.h>

#include "dg_common.cuh"
#include "dg_kernels_fp64.cuh"

namespace dgpf {

enum { VEL_UNIFORM = 0, VEL_RIDER_KOTHE = 1 };
// What a kinematic stage kernel writes: the right-hand side, or one stage of
// classical RK4 (w0: step start, acc: k1 + 2 k2 + 2 k3 so far).
enum KinMode { KIN_RHS = 0, KIN_K1 = 1, KIN_K2 = 2, KIN_K3 = 3, KIN_K4 = 4 };

// Constants of one triangle type of the split-rectangle mesh (dg_tri.cuh): det = d(x,y)/d(r,s),
// its inverse, the inverse-map derivatives, and per edge f the outward unit normal m, half the
// edge length and its reciprocal, the penalty eta_tri / h_e and the reference components of
// grad l . m (gr = rx m0 + ry m1, gs = sx m0 + sy m1).
struct TriConst {
  double det, idet, rx, ry, sx, sy;
  double m0[3], m1[3], hl[3], ihl[3], eta[3], gr[3], gs[3];
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
  const double *dt;        // device: the step size of the captured step sequences
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

// Spatial factor of the Rider-Kothe stream function, u = d(Psi)/dy and v = -d(Psi)/dx:
// Psi = sin^2(pi X) sin^2(pi Y) / pi.
__device__ __forceinline__ double kin_stream_factor(const KinParams &kp, double x, double y) {
  const double sx = sin(CUDART_PI * (x - kp.xc + 0.5)), sy = sin(CUDART_PI * (y - kp.yc + 0.5));
  return sx * sx * sy * sy / CUDART_PI;
}

// U at every node of the rectangles, [N][2]: a uniform field as given; the vortex as the
// discrete curl of its stream function at the element's nodes, U = sum_c Dy[j][c] Psi(i, c),
// V = -sum_c Dx[i][c] Psi(c, j) (Dx, Dy: the (2/h) D rows of the operator table).
template <int P>
__global__ void k_kin_velocity_table(const KinParams kp, double *__restrict__ tab) {
  constexpr int P1 = P + 1, NP = P1 * P1;
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const int e = (int)(n / NP), a = (int)(n % NP), i = a % P1, j = a / P1;
  const int ex = e % kp.nx, ey = e / kp.nx;
  const double x = kp.x0 + kp.hx * (ex + 0.5 * (__ldg(kp.xi + i) + 1.0));
  const double y = kp.y0 + kp.hy * (ey + 0.5 * (__ldg(kp.xi + j) + 1.0));
  if (kp.vel != VEL_RIDER_KOTHE) {
    kin_velocity_factor(kp, x, y, &tab[2 * n], &tab[2 * n + 1]);
    return;
  }
  const OpsLayout L{P1, NP};
  double U = 0.0, V = 0.0;
  for (int c = 0; c < P1; ++c) {
    const double xc = kp.x0 + kp.hx * (ex + 0.5 * (__ldg(kp.xi + c) + 1.0));
    const double yc = kp.y0 + kp.hy * (ey + 0.5 * (__ldg(kp.xi + c) + 1.0));
    U = fma(__ldg(kp.ops + L.Dy() + j * P1 + c), kin_stream_factor(kp, x, yc), U);
    V = fma(-__ldg(kp.ops + L.Dx() + i * P1 + c), kin_stream_factor(kp, xc, y), V);
  }
  tab[2 * n] = U;
  tab[2 * n + 1] = V;
}

template <int P>
cudaError_t launch_kin_velocity_table(const KinParams &kp, double *tab, cudaStream_t s) {
  k_kin_velocity_table<P><<<(unsigned)((kp.N + 255) / 256), 256, 0, s>>>(kp, tab);
  return cudaGetLastError();
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

// Node index of face node kk of face f (0 W, 1 E, 2 S, 3 N) in the x-fastest GLL order.
template <int P>
__device__ __forceinline__ int kin_face_node(int f, int kk) {
  constexpr int P1 = P + 1;
  return f == 0 ? kk * P1 : (f == 1 ? P + kk * P1 : (f == 2 ? kk : kk + P * P1));
}

// One stage of the kinematic mode in one launch: broken gradients, n, a_1,
// the volume term of -a_1 (D^ contractions) and the non-conservative
// transport at every node; at every face node the transport flux
// (lambda - m.u-) [[f]] and the SIP flux of a_1 with its lifted symmetric
// term, the neighbour's trace being evaluated here from its nodal values (a
// row of the neighbour's element), not read from a trace buffer; then M^-1
// and the right-hand side or an RK4 stage:
//   K1: acc = L,        out = w0 + dt/2 L
//   K2: acc += 2 L,     out = w0 + dt/2 L
//   K3: acc += 2 L,     out = w0 + dt L
//   K4: out = w0 + dt/6 (acc + L)   (out may be w0: each node is read, then
//                                    written, by the same thread)
// Neighbour values come from the stage input, which no stage writes, so the
// stages need no synchronisation beyond stream order.  The step size is read
// from device memory (*kp.dt), so captured step sequences serve any dt; the
// stage time is *kp.t0 + (kstep dt) + (frac dt), kstep the step's index in the
// captured sequence and frac the stage's fraction of the step (0, 1/2, 1/2, 1).
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_kin_stage(const KinParams kp, int mode, int kstep, double frac, const double *__restrict__ win,
            const double *w0, double *__restrict__ acc, double *out) {
  const double dt = __ldg(kp.dt);
  const double tstep = kstep * dt, toff = frac * dt;
  using G = Geom<P, 2, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  const OpsLayout L{P1, NP};
  __shared__ double s_op[4 * P1 * P1 + 3 * P1 + NP];
  __shared__ double s_f[2][EPB][NP];       // phi, psi; then -a_1
  __shared__ double s_nb[EPB][4][2][NP];   // the four neighbours' phi, psi
  __shared__ double s_tr[EPB][NP][6];      // phi, psi, d(phi)/dx, d(phi)/dy, n_x, n_y
  __shared__ double s_surf[EPB][NFK][2];
  __shared__ double s_lift[EPB][NFK];
  for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = kp.ops[t];
  const double *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy(), *Dhx = s_op + L.Dhx(), *Dhy = s_op + L.Dhy();
  const double *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const int N = kp.N;
  const bool act = lane && e < kp.E && in_bounds(kp.status, (long long)e * NP + a, N);
  const int i = a % P1, j = a / P1;
  const long n = (long)(act ? e : 0) * NP + a;
  const double2 *vt = reinterpret_cast<const double2 *>(kp.vel_tab);
  // The time factor of the velocity and dt/6, once per CTA: FP64 is this kernel's bound, and a
  // cosine or a division per thread would cost a fifth of its work.
  __shared__ double s_c[2];
  if (threadIdx.x == 0) {
    s_c[0] = kin_time_factor(kp, (*kp.t0 + tstep) + toff);
    s_c[1] = dt / 6.0;
  }

  const double phi = act ? __ldg(win + n) : 0.0, psi = act ? __ldg(win + N + n) : 0.0;
  const double2 U = __ldg(vt + n);
  if (lane) {
    s_f[0][le][a] = phi;
    s_f[1][le][a] = psi;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const long m = (long)(act ? kin_neighbour(kp, e, f) : 0) * NP + a;
      const bool ok = in_bounds(kp.status, m, N);
      s_nb[le][f][0][a] = ok ? __ldg(win + m) : 0.0;
      s_nb[le][f][1][a] = ok ? __ldg(win + N + m) : 0.0;
    }
  }
  __syncthreads();
  const double c = s_c[0], dt6 = s_c[1];
  const double u = U.x * c, v = U.y * c;
  double gpx = 0.0, gpy = 0.0, gsx = 0.0, gsy = 0.0;
#pragma unroll
  for (int k = 0; k < P1; ++k) {
    const double dx = Dx[i * P1 + k], dy = Dy[j * P1 + k];
    gpx = fma(dx, s_f[0][le][k + P1 * j], gpx);
    gsx = fma(dx, s_f[1][le][k + P1 * j], gsx);
    gpy = fma(dy, s_f[0][le][i + P1 * k], gpy);
    gsy = fma(dy, s_f[1][le][i + P1 * k], gsy);
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
    double *t = s_tr[le][a];
    t[0] = phi;
    t[1] = psi;
    t[2] = gpx;
    t[3] = gpy;
    t[4] = nx;
    t[5] = ny;
  }
  __syncthreads();
  double Rphi = 0.0;
#pragma unroll
  for (int k = 0; k < P1; ++k) {
    Rphi = fma(Dhx[i * P1 + k], s_f[0][le][k + P1 * j], Rphi);
    Rphi = fma(Dhy[j * P1 + k], s_f[1][le][i + P1 * k], Rphi);
  }
  Rphi -= u * gpx + v * gpy;
  const double Rpsi = -(u * gsx + v * gsy);

  // Face nodes: own trace from s_tr, the neighbour's from its nodal values.
  for (int t = a; t < NFK && lane; t += NP) {
    const int f = t / NK, kk = t % NK;
    const bool xf = f < 2;
    const double sg = (f & 1) ? 1.0 : -1.0;
    double flux = 0.0, fpsi = 0.0, lift = 0.0;
    if (act) {
      const int am = kin_face_node<P>(f, kk), ap = kin_face_node<P>(f ^ 1, kk);
      const int e2 = kin_neighbour(kp, e, f);
      const double *tm = s_tr[le][am];
      const double *nbp = s_nb[le][f][0], *nbs = s_nb[le][f][1];
      const int i2 = ap % P1, j2 = ap / P1;
      double qpx = 0.0, qpy = 0.0, qsx = 0.0, qsy = 0.0;  // the neighbour's gradients at its face node
#pragma unroll
      for (int k = 0; k < P1; ++k) {
        const double dx = Dx[i2 * P1 + k], dy = Dy[j2 * P1 + k];
        qpx = fma(dx, nbp[k + P1 * j2], qpx);
        qsx = fma(dx, nbs[k + P1 * j2], qsx);
        qpy = fma(dy, nbp[i2 + P1 * k], qpy);
        qsy = fma(dy, nbs[i2 + P1 * k], qsy);
      }
      const double q2 = qsx * qsx + qsy * qsy;
      double mx = 0.0, my = 0.0;
      if (q2 >= 1e-24) {
        const double r = rsqrt(q2);
        mx = qsx * r;
        my = qsy * r;
      }
      const long om = (long)e * NP + am, op = (long)e2 * NP + ap;
      const double2 Um = in_bounds(kp.status, om, N) ? __ldg(vt + om) : make_double2(0.0, 0.0);
      const double2 Up = in_bounds(kp.status, op, N) ? __ldg(vt + op) : make_double2(0.0, 0.0);
      const double phm = tm[0], psm = tm[1], php = nbp[ap], psp = nbs[ap];
      const double unm = (xf ? Um.x : Um.y) * c * sg, unp = (xf ? Up.x : Up.y) * c * sg;
      const double lam = fmax(fabs(unm), fabs(unp));
      const double wf = xf ? wfx[kk] : wfy[kk];
      const double eta = xf ? kp.eta_x : kp.eta_y;
      const double jump = php - phm;
      const double gn = 0.5 * ((xf ? qpx : qpy) + (xf ? tm[2] : tm[3])) * sg;
      const double sharp = 0.5 * (php * (1.0 - php) * (xf ? mx : my) + phm * (1.0 - phm) * (xf ? tm[4] : tm[5])) * sg;
      const double ahat = kp.Gamma * (kp.eps * (gn + eta * jump) - sharp);
      flux = wf * (lam - unm) * 0.5 * jump + wf * ahat;
      fpsi = wf * (lam - unm) * 0.5 * (psp - psm);
      lift = -wf * 0.5 * kp.Gamma * kp.eps * jump;
    }
    s_surf[le][t][0] = flux;
    s_surf[le][t][1] = fpsi;
    s_lift[le][t] = lift;
  }
  __syncthreads();
  if (!act) return;

  double sp = 0.0, ss = 0.0;
  if (i == 0) { sp += s_surf[le][0 * NK + j][0]; ss += s_surf[le][0 * NK + j][1]; }
  if (i == P) { sp += s_surf[le][1 * NK + j][0]; ss += s_surf[le][1 * NK + j][1]; }
  if (j == 0) { sp += s_surf[le][2 * NK + i][0]; ss += s_surf[le][2 * NK + i][1]; }
  if (j == P) { sp += s_surf[le][3 * NK + i][0]; ss += s_surf[le][3 * NK + i][1]; }
  sp += s_lift[le][0 * NK + j] * -Dx[0 * P1 + i] + s_lift[le][1 * NK + j] * Dx[P * P1 + i];
  sp += s_lift[le][2 * NK + i] * -Dy[0 * P1 + j] + s_lift[le][3 * NK + i] * Dy[P * P1 + j];
  const double im = invM[a];
  const double Lv[2] = {Rphi + sp * im, Rpsi + ss * im};
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
        r = base + dt6 * (acc[o] + Lv[vv]);
      }
    }
    bad |= !isfinite(r);
    out[o] = r;
  }
  if (kp.check_finite && bad) atomicOr(kp.status, STATUS_NONFINITE);
}

struct KinKernels {
  cudaError_t (*stage)(const KinParams &, int mode, int kstep, double frac, const double *win, const double *w0,
                       double *acc, double *out, cudaStream_t);
  cudaError_t (*velocity_table)(const KinParams &, double *tab, cudaStream_t);
};

template <int P>
cudaError_t launch_kin_stage(const KinParams &kp, int mode, int kstep, double frac, const double *win,
                             const double *w0, double *acc, double *out, cudaStream_t s) {
  using G = Geom<P, 2, false, false>;
  k_kin_stage<P><<<(kp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(kp, mode, kstep, frac, win, w0, acc, out);
  return cudaGetLastError();
}

bool kin_kernels(int p, KinKernels *out);

}  // namespace dgpf
