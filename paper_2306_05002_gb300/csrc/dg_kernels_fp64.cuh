// dg_kernels_fp64.cuh -- FP64 kernels of the DG right-hand side (GB300, sm_103a).
//
// Two kernels per right-hand side evaluation, both element-blocked (one CTA
// holds EPB whole elements, one thread per node):
//
//   k_volume   closure (stiffened gas, Sec. 2), broken gradients of phi and
//              psi (and u, v when viscous) by sum-factorised 1D contractions,
//              level-set normal n = grad psi/|grad psi|, a_1, curvature,
//              conservative fluxes, the weak-form volume term (tensor-product
//              Dhat contractions, Sec. 3 eq. "weakDG"), the non-conservative
//              transport -u.grad(phi) of Sec. 3 and the sources of Sec. 2.
//              Writes the volume part of M^-1 R and one trace record per face
//              node.
//   k_surface  per face node: Lax-Friedrichs flux, quasi-conservative
//              transport flux, SIP flux of a_1 and its derived terms, viscous
//              penalty flux (Sec. 3); lifts the SIP symmetric term along the
//              normal line; applies M^-1; adds the volume part; and writes
//              either L or one SSP-RK3 stage (fused update).
//
// On GB300 the FP64 pipe (about 0.5 TFMA/s) bounds this path, so the kernels
// spend FP64 instructions only on the scheme's arithmetic: operator tables
// are premultiplied by 2/h, index work is integer, and every division or
// square root is taken once per node.  The pressure is evaluated in the
// operation order of the stiffened-gas formula with explicit IEEE intrinsics
// (no FMA contraction): its recovery cancels ~4 digits against
// sum phi_l gamma_l Pinf_l/(gamma_l-1), and this keeps it reproducible.
#pragma once

#include "dg_common.cuh"

namespace dgpf {

// Block geometry of one kernel family.  EPBX > 0 overrides the number of
// elements per block (the batched kernels' tuned tile).
template <int P, int DIM, bool VISC, bool ST, int EPBX = 0>
struct Geom {
  static constexpr int P1 = P + 1;
  static constexpr int NP = DIM == 2 ? P1 * P1 : P1;
  static constexpr int NF = 2 * DIM;                 // faces per element
  static constexpr int NK = DIM == 2 ? P1 : 1;       // nodes per face
  static constexpr int NFK = NF * NK;                // face nodes per element
  // Elements per block: the smallest count that fills at least 60 threads with
  // under 7% of the last warp idle.  Small blocks spread a grid evenly over the
  // 152 SMs (the FP64 path is bound by the per-SM FP64 pipe, so balance, not
  // occupancy, decides its time).
  static constexpr int pick_epb() {
    for (int e = 1; e <= 64; ++e) {
      const int t = e * NP, tp = ((t + 31) / 32) * 32;
      if (t >= 60 && (tp - t) * 100 < 7 * tp) return e;
    }
    return (128 + NP - 1) / NP;
  }
  static constexpr int EPB = EPBX > 0 ? EPBX : pick_epb();
  static constexpr int THREADS = ((EPB * NP + 31) / 32) * 32;
  static constexpr int NT = VISC ? NT_VISCOUS : NT_INVISCID;
  static constexpr int NSTAGE = 12;                  // staged fields per node
  static constexpr int OPS = 4 * P1 * P1 + 3 * P1 + NP;  // operator table (OpsLayout) size
};

// Neighbour of element e across face f (0 W, 1 E, 2 S, 3 N), or -1 at a wall.
__device__ __forceinline__ int neighbour(const Params &p, int e, int f) {
  const int ex = e % p.nx, ey = e / p.nx;
  switch (f) {
    case 0: return ex > 0 ? e - 1 : (p.bc[0] == BC_PERIODIC ? e + p.nx - 1 : -1);
    case 1: return ex < p.nx - 1 ? e + 1 : (p.bc[1] == BC_PERIODIC ? e - p.nx + 1 : -1);
    case 2: return ey > 0 ? e - p.nx : (p.bc[2] == BC_PERIODIC ? e + p.nx * (p.ny - 1) : -1);
    default: return ey < p.ny - 1 ? e + p.nx : (p.bc[3] == BC_PERIODIC ? e - p.nx * (p.ny - 1) : -1);
  }
}

// Stiffened-gas pressure (Sec. 2), in the formula's own operation order:
//   rho e = rho E - (|rho u|^2 / 2) / rho
//   P = (rho e - (phi_1 C_1 + phi_2 C_2)) / (phi_1 g_1 + phi_2 g_2)
__device__ __forceinline__ double sg_pressure(const Params &p, double phi, double rho, double ru, double rv,
                                              double rE, double *Cm, double *den) {
  const double phi2 = __dsub_rn(1.0, phi);
  const double rhok = __ddiv_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(ru, ru), __dmul_rn(rv, rv))), rho);
  const double rhoe = __dsub_rn(rE, rhok);
  *Cm = __dadd_rn(__dmul_rn(phi, p.C1), __dmul_rn(phi2, p.C2));
  *den = __dadd_rn(__dmul_rn(phi, p.g1), __dmul_rn(phi2, p.g2));
  return __ddiv_rn(__dsub_rn(rhoe, *Cm), *den);
}

template <int P, int DIM, bool VISC, bool ST>
__global__ void __launch_bounds__(Geom<P, DIM, VISC, ST>::THREADS)
k_volume(const Params prm, const double *__restrict__ w, double *__restrict__ rvol, double *__restrict__ tr) {
  using G = Geom<P, DIM, VISC, ST>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int P11 = P1 * P1;
  __shared__ double s_op[4 * P11];
  __shared__ double s_f[G::NSTAGE][EPB][NP];

  for (int t = threadIdx.x; t < 4 * P11; t += blockDim.x) s_op[t] = prm.ops[t];
  const double *Dx = s_op, *Dy = s_op + P11, *Dhx = s_op + 2 * P11, *Dhy = s_op + 3 * P11;

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;  // padding lanes mirror the last element, write nothing
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const int N = prm.N;
  const bool act = lane && e < prm.E && in_bounds(prm.status, (long long)e * NP + a, N);
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const long n = (long)(act ? e : 0) * NP + a;

  double q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = act ? __ldg(w + (long)v * N + n) : (v == M1 || v == M2 ? 1.0 : 0.0);
  const double phi = q[PHI], psi = q[PSI];
  const double rho = q[M1] + q[M2];
  const double ir = 1.0 / rho;
  const double u = q[RU] * ir;
  const double v = DIM == 2 ? q[RV] * ir : 0.0;
  double Cm, den;
  const double Pr = sg_pressure(prm, phi, rho, q[RU], DIM == 2 ? q[RV] : 0.0, q[RE], &Cm, &den);
  const double B = fma(Pr, prm.Bp, prm.dC);
  const double k = 0.5 * (u * u + v * v);
  // Non-physical state: rho <= 0, a mixture 1/(gamma - 1) <= 0, or P + Pinf_mix <= 0, i.e.
  // P (1 + den) + Cm <= 0 with Pinf_mix = Cm / (1 + den) (Sec. 2 mixture rules).
  if (prm.check_finite && act && (rho <= 0.0 || den <= 0.0 || fma(Pr, den + 1.0, Cm) <= 0.0))
    atomicOr(prm.status, STATUS_NONPHYSICAL);

  if (lane) {
    s_f[0][le][a] = phi;
    s_f[1][le][a] = psi;
    if (VISC) {
      s_f[2][le][a] = u;
      s_f[3][le][a] = v;
    }
  }
  __syncthreads();

  // Broken gradients: sum-factorised contractions along the two GLL lines.
  double gpx = 0.0, gpy = 0.0, gsx = 0.0, gsy = 0.0, gux = 0.0, guy = 0.0, gvx = 0.0, gvy = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const double dx = Dx[i * P1 + c];
    const int ax = c + P1 * j;
    gpx = fma(dx, s_f[0][le][ax], gpx);
    gsx = fma(dx, s_f[1][le][ax], gsx);
    if (VISC) {
      gux = fma(dx, s_f[2][le][ax], gux);
      gvx = fma(dx, s_f[3][le][ax], gvx);
    }
    if (DIM == 2) {
      const double dy = Dy[j * P1 + c];
      const int ay = i + P1 * c;
      gpy = fma(dy, s_f[0][le][ay], gpy);
      gsy = fma(dy, s_f[1][le][ay], gsy);
      if (VISC) {
        guy = fma(dy, s_f[2][le][ay], guy);
        gvy = fma(dy, s_f[3][le][ay], gvy);
      }
    }
  }

  // The transport term keeps the broken gradients; with grad_lift the gradients of phi and psi
  // become BR1-lifted: at a face node, M^-1 w_f (f+ - f-) / 2 along the outward normal, f+ the
  // neighbour's value at the coincident node (none at walls and pressure boundaries).
  const double bpx = gpx, bpy = gpy, bsx = gsx, bsy = gsy;
  if (prm.grad_lift && act && (i == 0 || i == P || (DIM == 2 && (j == 0 || j == P)))) {
    const OpsLayout Lo{P1, NP};
    const double im = __ldg(prm.ops + Lo.invM() + a);
    auto lift = [&](int f, int kk, double &gx_phi, double &gx_psi, double sgn) {
      const int e2 = neighbour(prm, e, f);
      if (e2 < 0) return;
      const int f2 = f ^ 1;
      const int a2 = f2 == 0 ? P1 * kk : f2 == 1 ? P + P1 * kk : f2 == 2 ? kk : kk + P1 * P;
      const long n2 = (long)e2 * NP + a2;
      if (!in_bounds(prm.status, n2, N)) return;
      const double wf = DIM == 2 ? __ldg(prm.ops + (f < 2 ? Lo.wfx() : Lo.wfy()) + kk) : 1.0;
      const double c = sgn * 0.5 * im * wf;
      gx_phi += c * (__ldg(w + (long)PHI * N + n2) - phi);
      gx_psi += c * (__ldg(w + (long)PSI * N + n2) - psi);
    };
    const int kx = DIM == 2 ? j : 0;
    if (i == 0) lift(0, kx, gpx, gsx, -1.0);
    if (i == P) lift(1, kx, gpx, gsx, 1.0);
    if (DIM == 2 && j == 0) lift(2, i, gpy, gsy, -1.0);
    if (DIM == 2 && j == P) lift(3, i, gpy, gsy, 1.0);
  }

  // Interface normal from the level set (zero where |grad psi| < 1e-12).
  const double g2 = gsx * gsx + gsy * gsy;
  double nx = 0.0, ny = 0.0;
  if (g2 >= 1e-24) {
    const double r = rsqrt(g2);
    nx = gsx * r;
    ny = gsy * r;
  }
  const double sphi = phi * (1.0 - phi);
  const double a1x = prm.Gamma * (prm.eps * gpx - sphi * nx);
  const double a1y = prm.Gamma * (prm.eps * gpy - sphi * ny);

  // Viscous stress tau = 2 mu (S - div(u)/3 I), mixture mu.
  double txx = 0.0, txy = 0.0, tyy = 0.0, mu = 0.0;
  if (VISC) {
    mu = prm.mu1 * phi + prm.mu2 * (1.0 - phi);
    const double div3 = (gux + gvy) * (1.0 / 3.0);
    txx = 2.0 * mu * (gux - div3);
    tyy = 2.0 * mu * (gvy - div3);
    txy = mu * (guy + gvx);
  }

  // Curvature kappa = -div n from the nodal normal.
  double kappa = 0.0;
  if (ST) {
    if (lane) {
      s_f[4][le][a] = nx;
      s_f[5][le][a] = ny;
    }
    __syncthreads();
    double dv = 0.0;
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      dv = fma(Dx[i * P1 + c], s_f[4][le][c + P1 * j], dv);
      if (DIM == 2) dv = fma(Dy[j * P1 + c], s_f[5][le][i + P1 * c], dv);
    }
    kappa = -dv;
  }

  // Conservative fluxes (moved to the right-hand side), per equation.
  const double cE = prm.drho0 * k + B;  // coefficient of a_1 in the energy flux
  double F[G::NSTAGE];
  F[0] = -a1x;
  F[1] = -a1y;
  F[2] = q[M1] * u - prm.rho01 * a1x;
  F[3] = q[M1] * v - prm.rho01 * a1y;
  F[4] = q[M2] * u + prm.rho02 * a1x;
  F[5] = q[M2] * v + prm.rho02 * a1y;
  F[6] = q[RU] * u + Pr - prm.drho0 * a1x * u - txx;
  F[7] = q[RU] * v - prm.drho0 * a1y * u - txy;
  F[8] = q[RV] * u - prm.drho0 * a1x * v - txy;
  F[9] = q[RV] * v + Pr - prm.drho0 * a1y * v - tyy;
  F[10] = (q[RE] + Pr) * u - cE * a1x - (txx * u + txy * v);
  F[11] = (q[RE] + Pr) * v - cE * a1y - (txy * u + tyy * v);
  __syncthreads();
  if (lane) {
#pragma unroll
    for (int s = 0; s < G::NSTAGE; ++s) s_f[s][le][a] = F[s];
  }
  __syncthreads();

  // Volume term: M^-1 sum_k w_k J grad(l_a)(x_k) . F_k = Dhx F^x + Dhy F^y.
  double R[NV];
#pragma unroll
  for (int eq = 0; eq < 6; ++eq) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      acc = fma(Dhx[i * P1 + c], s_f[2 * eq][le][c + P1 * j], acc);
      if (DIM == 2) acc = fma(Dhy[j * P1 + c], s_f[2 * eq + 1][le][i + P1 * c], acc);
    }
    R[eq == 0 ? PHI : eq + 1] = acc;
  }
  // Non-conservative transport of phi and psi (Sec. 3: treated as a source), broken gradients.
  R[PHI] -= u * bpx + v * bpy;
  R[PSI] = -(u * bsx + v * bsy);
  if (prm.gravity) {
    R[RU] += rho * prm.gx;
    R[RV] += rho * prm.gy;
    R[RE] += rho * (prm.gx * u + prm.gy * v);
  }
  if (ST) {
    // CSF surface tension sigma kappa n delta, delta = |grad phi|.
    const double s = prm.sigma * kappa * sqrt(gpx * gpx + gpy * gpy);
    R[RU] += s * nx;
    R[RV] += s * ny;
    R[RE] += s * (u * nx + v * ny);
  }
  if (act) {
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) rvol[(long)vv * N + n] = R[vv];
  }

  // Face traces.
  const bool onW = i == 0, onE = i == P;
  const bool onS = DIM == 2 && j == 0, onN = DIM == 2 && j == P;
  if (act && (onW || onE || onS || onN)) {
    const double c = sqrt((Pr + (Pr + Cm) / den) * ir);  // mixture sound speed
    const double tx[NT_VISCOUS] = {phi, psi, q[M1], q[M2], q[RU], q[RV], q[RE], u, v, Pr, c, B,
                                   0.0, 0.0, 0.0, 0.0, mu};
    const long base = (long)e * NFK;
    const long stride = (long)prm.E * NFK;
    auto put = [&](int f, int kk, double gn, double nn, double t1, double t2) {
      const long o = base + f * NK + kk;
      if (!in_bounds(prm.status, o, stride)) return;
#pragma unroll
      for (int qf = 0; qf < T_GPHI; ++qf) tr[qf * stride + o] = tx[qf];
      tr[T_GPHI * stride + o] = gn;
      tr[T_N * stride + o] = nn;
      if (VISC) {
        tr[T_TX * stride + o] = t1;
        tr[T_TY * stride + o] = t2;
        tr[T_MU * stride + o] = mu;
      }
    };
    const int kx = DIM == 2 ? j : 0;
    if (onW) put(0, kx, gpx, nx, txx, txy);
    if (onE) put(1, kx, gpx, nx, txx, txy);
    if (onS) put(2, i, gpy, ny, txy, tyy);
    if (onN) put(3, i, gpy, ny, txy, tyy);
  }
}

template <int P, int DIM, bool VISC, bool ST>
__global__ void __launch_bounds__(Geom<P, DIM, VISC, ST>::THREADS)
k_surface(const Params prm, int mode, double dt, const double *__restrict__ w0, const double *__restrict__ ws,
          const double *__restrict__ rvol, const double *__restrict__ tr, double *__restrict__ out) {
  using G = Geom<P, DIM, VISC, ST>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK, NT = G::NT;
  constexpr int P11 = P1 * P1;
  const OpsLayout L{P1, NP};
  __shared__ double s_op[4 * P11 + 3 * P1 + NP];
  __shared__ double s_surf[EPB][NFK][NV];
  __shared__ double s_lift[EPB][NFK][6];

  for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = prm.ops[t];
  __syncthreads();
  const double *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy();
  const double *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const bool act = lane && e < prm.E;
  const long stride = (long)prm.E * NFK;

  // Phase 1: numerical fluxes at the element's face nodes.
  for (int t = a; t < NFK && lane; t += NP) {
    const int f = t / NK, kk = t % NK;
    const int e2 = act ? neighbour(prm, e, f) : -1;
    const bool wall = e2 < 0;
    const bool xf = f < 2;
    const double sg = (f & 1) ? 1.0 : -1.0;  // m = sg * e_axis
    double Tm[NT], Tp[NT];
    const long om = (long)(act ? e : 0) * NFK + t;
    const bool okm = act && in_bounds(prm.status, om, stride);
#pragma unroll
    for (int qf = 0; qf < NT; ++qf) Tm[qf] = okm ? __ldg(tr + qf * stride + om) : (qf == T_M1 ? 1.0 : 0.0);
    if (!wall) {
      const long op = (long)e2 * NFK + (f ^ 1) * NK + kk;
      const bool okp = in_bounds(prm.status, op, stride);
#pragma unroll
      for (int qf = 0; qf < NT; ++qf) Tp[qf] = okp ? __ldg(tr + qf * stride + op) : Tm[qf];
    } else {
#pragma unroll
      for (int qf = 0; qf < NT; ++qf) Tp[qf] = Tm[qf];
      const int bc = prm.bc[f];
      if (bc == BC_SLIP) {  // reverse the normal component only
        if (xf) { Tp[T_RU] = -Tm[T_RU]; Tp[T_U] = -Tm[T_U]; }
        else    { Tp[T_RV] = -Tm[T_RV]; Tp[T_V] = -Tm[T_V]; }
      } else if (bc == BC_PRESSURE) {
        // exterior state: own phase field and partial densities, at rest, at p_bc;
        // rho E from the stiffened-gas relation, then the closure of that state
        const double phi = Tm[T_PHI], phi2 = __dsub_rn(1.0, phi);
        const double den0 = __dadd_rn(__dmul_rn(phi, prm.g1), __dmul_rn(phi2, prm.g2));
        const double Cm0 = __dadd_rn(__dmul_rn(phi, prm.C1), __dmul_rn(phi2, prm.C2));
        const double rho = Tm[T_M1] + Tm[T_M2];
        Tp[T_RU] = Tp[T_RV] = Tp[T_U] = Tp[T_V] = 0.0;
        Tp[T_RE] = __dadd_rn(__dmul_rn(prm.p_bc[f], den0), Cm0);
        double Cm, den;
        const double Pg = sg_pressure(prm, phi, rho, 0.0, 0.0, Tp[T_RE], &Cm, &den);
        Tp[T_P] = Pg;
        Tp[T_C] = sqrt((Pg + (Pg + Cm) / den) / rho);
        Tp[T_B] = fma(Pg, prm.Bp, prm.dC);
      } else {              // no-slip: reverse the velocity
        Tp[T_RU] = -Tm[T_RU]; Tp[T_U] = -Tm[T_U];
        Tp[T_RV] = -Tm[T_RV]; Tp[T_V] = -Tm[T_V];
      }
    }
    const double mx = xf ? sg : 0.0, my = xf ? 0.0 : sg;
    const double unm = Tm[T_U] * mx + Tm[T_V] * my;
    const double unp = Tp[T_U] * mx + Tp[T_V] * my;
    const double lam = fmax(fabs(unm) + Tm[T_C], fabs(unp) + Tp[T_C]);
    const double wf = xf ? wfx[kk] : wfy[kk];

    double S[NV];
    // Lax-Friedrichs flux {F}.m - lambda [[w]], [[w]] = (w+ - w-)/2.
    {
      const double Fm[5] = {Tm[T_M1] * unm, Tm[T_M2] * unm, Tm[T_RU] * unm + Tm[T_P] * mx,
                            Tm[T_RV] * unm + Tm[T_P] * my, (Tm[T_RE] + Tm[T_P]) * unm};
      const double Fp[5] = {Tp[T_M1] * unp, Tp[T_M2] * unp, Tp[T_RU] * unp + Tp[T_P] * mx,
                            Tp[T_RV] * unp + Tp[T_P] * my, (Tp[T_RE] + Tp[T_P]) * unp};
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const int vv = M1 + c;
        S[vv] = -wf * (0.5 * (Fp[c] + Fm[c]) - lam * 0.5 * (Tp[vv] - Tm[vv]));
      }
    }
    // Quasi-conservative transport: (lambda - m.u-) [[phi]], same for psi.
    S[PHI] = wf * (lam - unm) * 0.5 * (Tp[T_PHI] - Tm[T_PHI]);
    S[PSI] = wf * (lam - unm) * 0.5 * (Tp[T_PSI] - Tm[T_PSI]);

    double lift[6] = {0, 0, 0, 0, 0, 0};
    if (!wall) {
      // SIP flux of a_1: Gamma [eps ({grad phi}.m + eta (phi+ - phi-)) - {phi(1-phi) n}.m]
      const double eta = xf ? prm.eta_x : prm.eta_y;
      const double jump = Tp[T_PHI] - Tm[T_PHI];
      const double gn = 0.5 * (Tp[T_GPHI] + Tm[T_GPHI]) * sg;
      const double sharp = 0.5 * (Tp[T_PHI] * (1.0 - Tp[T_PHI]) * Tp[T_N] + Tm[T_PHI] * (1.0 - Tm[T_PHI]) * Tm[T_N]) * sg;
      const double ahat = prm.Gamma * (prm.eps * (gn + eta * jump) - sharp);
      const double km = 0.5 * (Tm[T_U] * Tm[T_U] + Tm[T_V] * Tm[T_V]);
      const double kp = 0.5 * (Tp[T_U] * Tp[T_U] + Tp[T_V] * Tp[T_V]);
      // face coefficients of the a_1-derived terms
      const double Cq[6] = {1.0, prm.rho01, -prm.rho02, prm.drho0 * 0.5 * (Tp[T_U] + Tm[T_U]),
                            prm.drho0 * 0.5 * (Tp[T_V] + Tm[T_V]),
                            0.5 * (Tp[T_B] + Tm[T_B]) + prm.drho0 * 0.5 * (kp + km)};
      const double sym = -wf * 0.5 * prm.Gamma * prm.eps * jump;
      const int slot[6] = {PHI, M1, M2, RU, RV, RE};
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        S[slot[c]] += wf * Cq[c] * ahat;
        lift[c] = Cq[c] * sym;
      }
    }
    if (VISC) {
      const double eta = xf ? prm.eta_x : prm.eta_y;
      const double mua = 0.5 * (Tp[T_MU] + Tm[T_MU]);
      const double tmx = Tm[T_TX] * sg, tmy = Tm[T_TY] * sg;  // tau- . m
      const double tpx = Tp[T_TX] * sg, tpy = Tp[T_TY] * sg;  // tau+ . m
      S[RU] += wf * (0.5 * (tpx + tmx) + eta * mua * (Tp[T_U] - Tm[T_U]));
      S[RV] += wf * (0.5 * (tpy + tmy) + eta * mua * (Tp[T_V] - Tm[T_V]));
      const double km = 0.5 * (Tm[T_U] * Tm[T_U] + Tm[T_V] * Tm[T_V]);
      const double kp = 0.5 * (Tp[T_U] * Tp[T_U] + Tp[T_V] * Tp[T_V]);
      const double tum = tmx * Tm[T_U] + tmy * Tm[T_V];
      const double tup = tpx * Tp[T_U] + tpy * Tp[T_V];
      S[RE] += wf * (0.5 * (tup + tum) + eta * mua * (kp - km));
    }
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) s_surf[le][t][vv] = S[vv];
#pragma unroll
    for (int c = 0; c < 6; ++c) s_lift[le][t][c] = lift[c];
  }
  __syncthreads();

  // Phase 2: gather onto the element's nodes, lift the symmetric term along
  // the normal lines, apply M^-1, add the volume part, write L or the stage.
  if (!act || !in_bounds(prm.status, (long long)e * NP + a, prm.N)) return;
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  double acc[NV] = {0, 0, 0, 0, 0, 0, 0};
  auto face_add = [&](int f, int kk) {
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) acc[vv] += s_surf[le][f * NK + kk][vv];
  };
  const int kx = DIM == 2 ? j : 0;
  if (i == 0) face_add(0, kx);
  if (i == P) face_add(1, kx);
  if (DIM == 2 && j == 0) face_add(2, i);
  if (DIM == 2 && j == P) face_add(3, i);
  {
    const int slot[6] = {PHI, M1, M2, RU, RV, RE};
    const double lw = -Dx[0 * P1 + i], le_ = Dx[P * P1 + i];
#pragma unroll
    for (int c = 0; c < 6; ++c)
      acc[slot[c]] += s_lift[le][0 * NK + kx][c] * lw + s_lift[le][1 * NK + kx][c] * le_;
    if (DIM == 2) {
      const double ls = -Dy[0 * P1 + j], ln = Dy[P * P1 + j];
#pragma unroll
      for (int c = 0; c < 6; ++c)
        acc[slot[c]] += s_lift[le][2 * NK + i][c] * ls + s_lift[le][3 * NK + i][c] * ln;
    }
  }
  const double im = invM[a];
  const long n = (long)e * NP + a;
  const int N = prm.N;
  if (prm.dt_dev) dt = __ldg(prm.dt_dev);
  bool bad = false;
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) {
    const long o = (long)vv * N + n;
    const double Lv = __ldg(rvol + o) + acc[vv] * im;
    double r;
    if (mode == MODE_RHS) {
      r = Lv;
    } else {
      const double st = fma(dt, Lv, __ldg(ws + o));
      if (mode == MODE_S1) r = st;
      else if (mode == MODE_S2) r = 0.75 * __ldg(w0 + o) + 0.25 * st;
      else r = (1.0 / 3.0) * __ldg(w0 + o) + (2.0 / 3.0) * st;
    }
    bad |= !isfinite(r);
    out[o] = r;
  }
  if (prm.check_finite && bad) atomicOr(prm.status, STATUS_NONFINITE);
}

template <int P, int DIM, bool VISC, bool ST>
cudaError_t launch_volume(const Params &prm, const double *w, double *rvol, double *trace, cudaStream_t s) {
  using G = Geom<P, DIM, VISC, ST>;
  const int blocks = (prm.E + G::EPB - 1) / G::EPB;
  k_volume<P, DIM, VISC, ST><<<blocks, G::THREADS, 0, s>>>(prm, w, rvol, trace);
  return cudaGetLastError();
}

template <int P, int DIM, bool VISC, bool ST>
cudaError_t launch_surface(const Params &prm, int mode, double dt, const double *w0, const double *ws,
                           const double *rvol, const double *trace, double *out, cudaStream_t s) {
  using G = Geom<P, DIM, VISC, ST>;
  const int blocks = (prm.E + G::EPB - 1) / G::EPB;
  k_surface<P, DIM, VISC, ST><<<blocks, G::THREADS, 0, s>>>(prm, mode, dt, w0, ws, rvol, trace, out);
  return cudaGetLastError();
}

template <int P, int DIM, bool VISC, bool ST>
KernelSet make_set() {
  using G = Geom<P, DIM, VISC, ST>;
  return KernelSet{&launch_volume<P, DIM, VISC, ST>, &launch_surface<P, DIM, VISC, ST>, G::NT, G::EPB, G::THREADS};
}

// All families of one order.
template <int P>
bool kernels_fp64_p(int dim, bool viscous, bool st, KernelSet *out) {
  if (dim == 1) {
    if (viscous || st) return false;
    *out = make_set<P, 1, false, false>();
    return true;
  }
  if (!viscous && !st) *out = make_set<P, 2, false, false>();
  else if (viscous && !st) *out = make_set<P, 2, true, false>();
  else if (!viscous && st) *out = make_set<P, 2, false, true>();
  else *out = make_set<P, 2, true, true>();
  return true;
}

}  // namespace dgpf
