// dg_reinit.cuh -- level-set re-initialisation (end of Sec. 3), FP64.
//
// In pseudo-time tau, from psi0 = phi - 1/2:
//   d(psi)/d(tau) = S (1 - |grad psi|) + div(nu grad psi),   S = tanh(psi0 / (2 eps |grad psi0|)),
// the hyperbolic term a nodal source on the broken gradient, the diffusion
// with the SIP flux nu ({grad psi}.m + eta (psi+ - psi-)) and its lifted
// symmetric term (no flux through walls), three-stage SSP Runge-Kutta.  The
// sign of the hyperbolic term is the one under which |grad psi| relaxes to 1
// (printed with the opposite sign, it grows at the interface).  Only psi
// changes; phi and every other field of the state are left as they are.
#pragma once

#include "dg_common.cuh"
#include "dg_kernels_fp64.cuh"

namespace dgpf {

struct ReinitParams {
  int nx, ny, E, N;
  int bc[4];
  double eps, nu;
  double eta_x, eta_y;
  const double *ops;  // operator table (OpsLayout)
  unsigned *status;   // the context's status word (the bounds-checked build latches STATUS_BOUNDS)
};

__device__ __forceinline__ int ri_neighbour(const ReinitParams &rp, int e, int f) {
  const int ex = e % rp.nx, ey = e / rp.nx;
  switch (f) {
    case 0: return ex > 0 ? e - 1 : (rp.bc[0] == BC_PERIODIC ? e + rp.nx - 1 : -1);
    case 1: return ex < rp.nx - 1 ? e + 1 : (rp.bc[1] == BC_PERIODIC ? e - rp.nx + 1 : -1);
    case 2: return ey > 0 ? e - rp.nx : (rp.bc[2] == BC_PERIODIC ? e + rp.nx * (rp.ny - 1) : -1);
    default: return ey < rp.ny - 1 ? e + rp.nx : (rp.bc[3] == BC_PERIODIC ? e - rp.nx * (rp.ny - 1) : -1);
  }
}

// Broken gradient of the shared-memory field f of element slot le at node (i, j).
template <int P1, int DIM, int EPB, int NP>
__device__ __forceinline__ void ri_grad(const double *Dx, const double *Dy, const double (*f)[NP], int le, int i,
                                        int j, double *gx, double *gy) {
  double sx = 0.0, sy = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    sx = fma(Dx[i * P1 + c], f[le][c + P1 * j], sx);
    if (DIM == 2) sy = fma(Dy[j * P1 + c], f[le][i + P1 * c], sy);
  }
  *gx = sx;
  *gy = sy;
}

// Smeared sign S from psi0 = phi - 1/2 (S = sign(psi0) where |grad psi0| < 1e-12),
// and psi <- psi0.  w: the state, phi at w[0..N), psi at w[N..2N).
template <int P, int DIM>
__global__ void __launch_bounds__(Geom<P, DIM, false, false>::THREADS)
k_ri_sign(const ReinitParams rp, double *w, double *S) {
  using G = Geom<P, DIM, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, P11 = P1 * P1;
  __shared__ double s_op[2 * P11];
  __shared__ double s_f[EPB][NP];
  for (int t = threadIdx.x; t < 2 * P11; t += blockDim.x) s_op[t] = rp.ops[t];
  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < rp.E && in_bounds(rp.status, (long long)e * NP + a, rp.N);
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const long n = (long)(act ? e : 0) * NP + a;
  const double p0 = act ? w[n] - 0.5 : 0.0;
  if (lane) s_f[le][a] = p0;
  __syncthreads();
  double gx, gy;
  ri_grad<P1, DIM, EPB, NP>(s_op, s_op + P11, s_f, le, i, j, &gx, &gy);
  const double gm = sqrt(gx * gx + gy * gy);
  const double sg = (gm < 1e-12 || !(rp.eps > 0.0)) ? (p0 > 0.0 ? 1.0 : (p0 < 0.0 ? -1.0 : 0.0))
                                                    : tanh(p0 / (2.0 * rp.eps * gm));
  if (act) {
    S[n] = sg;
    w[rp.N + n] = p0;
  }
}

// Volume part: S (1 - |grad psi|) + M^-1 int grad l . (-nu grad psi), and the traces (psi, d psi / d axis).
template <int P, int DIM>
__global__ void __launch_bounds__(Geom<P, DIM, false, false>::THREADS)
k_ri_volume(const ReinitParams rp, const double *__restrict__ psi, const double *__restrict__ S,
            double *__restrict__ rvol, double *__restrict__ tr) {
  using G = Geom<P, DIM, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK, P11 = P1 * P1;
  __shared__ double s_op[4 * P11];
  __shared__ double s_f[2][EPB][NP];
  for (int t = threadIdx.x; t < 4 * P11; t += blockDim.x) s_op[t] = rp.ops[t];
  const double *Dx = s_op, *Dy = s_op + P11, *Dhx = s_op + 2 * P11, *Dhy = s_op + 3 * P11;
  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < rp.E && in_bounds(rp.status, (long long)e * NP + a, rp.N);
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const long n = (long)(act ? e : 0) * NP + a;
  const double ps = act ? __ldg(psi + n) : 0.0;
  if (lane) s_f[0][le][a] = ps;
  __syncthreads();
  double gx, gy;
  ri_grad<P1, DIM, EPB, NP>(Dx, Dy, s_f[0], le, i, j, &gx, &gy);
  if (lane) {
    s_f[0][le][a] = -rp.nu * gx;
    s_f[1][le][a] = -rp.nu * gy;
  }
  __syncthreads();
  double R = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    R = fma(Dhx[i * P1 + c], s_f[0][le][c + P1 * j], R);
    if (DIM == 2) R = fma(Dhy[j * P1 + c], s_f[1][le][i + P1 * c], R);
  }
  R += (act ? __ldg(S + n) : 0.0) * (1.0 - sqrt(gx * gx + gy * gy));
  if (act) rvol[n] = R;
  const bool onW = i == 0, onE = i == P, onS = DIM == 2 && j == 0, onN = DIM == 2 && j == P;
  if (act && (onW || onE || onS || onN)) {
    const long base = (long)e * NFK, stride = (long)rp.E * NFK;
    auto put = [&](int f, int kk, double gn) {
      if (!in_bounds(rp.status, base + f * NK + kk, stride)) return;
      tr[base + f * NK + kk] = ps;
      tr[stride + base + f * NK + kk] = gn;
    };
    const int kx = DIM == 2 ? j : 0;
    if (onW) put(0, kx, gx);
    if (onE) put(1, kx, gx);
    if (onS) put(2, i, gy);
    if (onN) put(3, i, gy);
  }
}

// Surface part: SIP flux and lifted symmetric term, M^-1, and one SSP-RK3
// stage of psi (mode MODE_S1..S3; out may be w0: each node is read, then
// written, by the same thread).
template <int P, int DIM>
__global__ void __launch_bounds__(Geom<P, DIM, false, false>::THREADS)
k_ri_surface(const ReinitParams rp, int mode, double dtau, const double *w0, const double *__restrict__ ws,
             const double *__restrict__ rvol, const double *__restrict__ tr, double *out) {
  using G = Geom<P, DIM, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  const OpsLayout L{P1, NP};
  __shared__ double s_op[4 * P1 * P1 + 3 * P1 + NP];
  __shared__ double s_surf[EPB][NFK];
  __shared__ double s_lift[EPB][NFK];
  for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = rp.ops[t];
  __syncthreads();
  const double *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy();
  const double *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();
  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < rp.E && in_bounds(rp.status, (long long)e * NP + a, rp.N);
  const long stride = (long)rp.E * NFK;
  for (int t = a; t < NFK && lane; t += NP) {
    const int f = t / NK, kk = t % NK;
    const int e2 = act ? ri_neighbour(rp, e, f) : -1;
    double flux = 0.0, lift = 0.0;
    const long om = (long)(act ? e : 0) * NFK + t, op = (long)(e2 >= 0 ? e2 : 0) * NFK + (f ^ 1) * NK + kk;
    if (e2 >= 0 && in_bounds(rp.status, om, stride) && in_bounds(rp.status, op, stride)) {
      const double sg = (f & 1) ? 1.0 : -1.0;
      const double jump = __ldg(tr + op) - __ldg(tr + om);
      const double gn = 0.5 * (__ldg(tr + stride + op) + __ldg(tr + stride + om)) * sg;
      const double wf = f < 2 ? wfx[kk] : wfy[kk];
      const double eta = f < 2 ? rp.eta_x : rp.eta_y;
      flux = wf * rp.nu * (gn + eta * jump);
      lift = -wf * 0.5 * rp.nu * jump;
    }
    s_surf[le][t] = flux;
    s_lift[le][t] = lift;
  }
  __syncthreads();
  if (!act) return;
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const int kx = DIM == 2 ? j : 0;
  double acc = 0.0;
  if (i == 0) acc += s_surf[le][0 * NK + kx];
  if (i == P) acc += s_surf[le][1 * NK + kx];
  if (DIM == 2 && j == 0) acc += s_surf[le][2 * NK + i];
  if (DIM == 2 && j == P) acc += s_surf[le][3 * NK + i];
  acc += s_lift[le][0 * NK + kx] * -Dx[0 * P1 + i] + s_lift[le][1 * NK + kx] * Dx[P * P1 + i];
  if (DIM == 2) acc += s_lift[le][2 * NK + i] * -Dy[0 * P1 + j] + s_lift[le][3 * NK + i] * Dy[P * P1 + j];
  const long n = (long)e * NP + a;
  const double Lv = __ldg(rvol + n) + acc * invM[a];
  const double st = fma(dtau, Lv, __ldg(ws + n));
  double r;
  if (mode == MODE_RHS) r = Lv;
  else if (mode == MODE_S1) r = st;
  else if (mode == MODE_S2) r = 0.75 * w0[n] + 0.25 * st;
  else r = (1.0 / 3.0) * w0[n] + (2.0 / 3.0) * st;
  out[n] = r;
}

template <int P, int DIM>
cudaError_t launch_ri_sign(const ReinitParams &rp, double *w, double *S, cudaStream_t s) {
  using G = Geom<P, DIM, false, false>;
  k_ri_sign<P, DIM><<<(rp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(rp, w, S);
  return cudaGetLastError();
}

template <int P, int DIM>
cudaError_t launch_ri_volume(const ReinitParams &rp, const double *psi, const double *S, double *rvol, double *tr,
                             cudaStream_t s) {
  using G = Geom<P, DIM, false, false>;
  k_ri_volume<P, DIM><<<(rp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(rp, psi, S, rvol, tr);
  return cudaGetLastError();
}

template <int P, int DIM>
cudaError_t launch_ri_surface(const ReinitParams &rp, int mode, double dtau, const double *w0, const double *ws,
                              const double *rvol, const double *tr, double *out, cudaStream_t s) {
  using G = Geom<P, DIM, false, false>;
  k_ri_surface<P, DIM><<<(rp.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(rp, mode, dtau, w0, ws, rvol, tr, out);
  return cudaGetLastError();
}

struct ReinitKernels {
  cudaError_t (*sign)(const ReinitParams &, double *w, double *S, cudaStream_t);
  cudaError_t (*volume)(const ReinitParams &, const double *psi, const double *S, double *rvol, double *tr,
                        cudaStream_t);
  cudaError_t (*surface)(const ReinitParams &, int mode, double dtau, const double *w0, const double *ws,
                         const double *rvol, const double *tr, double *out, cudaStream_t);
  int nfk;
};

bool reinit_kernels(int p, int dim, ReinitKernels *out);

}  // namespace dgpf
