// dg_adjoint.cuh -- discrete adjoint (vector-Jacobian product) of the FP64
// right-hand side, for the inviscid equations without surface tension
// (gravity allowed): mu = (dL/dw)^T lambda, written by hand in reverse mode.
//
// Three launches per product:
//   k_volume      (forward, dg_kernels_fp64.cuh) -- the face traces of w;
//   k_adj_face    per element face node: the adjoint of the trace record,
//                 from the numerical fluxes of both elements sharing the face;
//   k_adj_volume  per element: recomputes the node quantities and runs the
//                 reverse of fluxes, a_1, normal, gradients and closure, adds
//                 the trace adjoints, and writes
//                 out = a x + b mu + c y + d z   (fused combination used by
//                 the reverse of the SSP-RK3 stages).
//
// Face adjoints.  The Lax-Friedrichs fluxes and the SIP flux of every
// a_1-derived term are conservative: seen from the neighbour (normal -m, the
// two traces swapped) their contribution is the negative of the own one,
// with the same lambda.  So the two elements' contributions to the adjoint of
// one trace come from one reverse evaluation seeded with (own seed -
// neighbour seed); only the non-conservative transport terms of phi and psi
// are reversed from both sides.  Where the two one-sided speeds tie in
// lambda = max(|u-.m| + c-, |u+.m| + c+) the derivative is given to the own
// side (a set of measure zero: the jump there is what lambda multiplies).
#pragma once

#include "dg_kernels_fp64.cuh"

namespace dgpf {

// Node index of face node k on face f.
template <int P, int DIM>
__device__ __forceinline__ int face_node(int f, int k) {
  constexpr int P1 = P + 1;
  if (DIM == 1) return f == 0 ? 0 : P;
  switch (f) {
    case 0: return P1 * k;
    case 1: return P + P1 * k;
    case 2: return k;
    default: return k + P1 * P;
  }
}

// Seeds of one element's face evaluation at face node (f, k): the adjoint of
// its surface contributions (lambda M^-1 at the face node) and of its lift
// coefficients (sum over the normal line of lambda M^-1 grad(l_b).m).
template <int P, int DIM>
__device__ __forceinline__ void face_seeds(const double *__restrict__ lam, int N, int e, int f, int k,
                                           const double *Dx, const double *Dy, const double *invM, double sS[NV],
                                           double sL[6]) {
  constexpr int P1 = P + 1, NP = DIM == 2 ? P1 * P1 : P1;
  const long base = (long)e * NP;
  const int a = face_node<P, DIM>(f, k);
#pragma unroll
  for (int v = 0; v < NV; ++v) sS[v] = __ldg(lam + (long)v * N + base + a) * invM[a];
  const int slot[6] = {PHI, M1, M2, RU, RV, RE};
#pragma unroll
  for (int c = 0; c < 6; ++c) sL[c] = 0.0;
  for (int l = 0; l < P1; ++l) {
    int b;
    double g;
    if (f < 2) {  // line along x through row k
      b = DIM == 2 ? l + P1 * k : l;
      g = f == 0 ? -Dx[0 * P1 + l] : Dx[P * P1 + l];
    } else {      // line along y through column k
      b = k + P1 * l;
      g = f == 2 ? -Dy[0 * P1 + l] : Dy[P * P1 + l];
    }
    const double wgt = g * invM[b];
#pragma unroll
    for (int c = 0; c < 6; ++c) sL[c] += __ldg(lam + (long)slot[c] * N + base + b) * wgt;
  }
}

template <int P, int DIM>
__global__ void __launch_bounds__(Geom<P, DIM, false, false>::THREADS)
k_adj_face(const Params prm, const double *__restrict__ lam, const double *__restrict__ tr,
           double *__restrict__ trbar) {
  using G = Geom<P, DIM, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int NT = NT_INVISCID;
  const OpsLayout L{P1, NP};
  __shared__ double s_op[4 * P1 * P1 + 3 * P1 + NP];
  for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = prm.ops[t];
  __syncthreads();
  const double *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy();
  const double *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();

  const int le = threadIdx.x / NP, a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  if (le >= EPB || e >= prm.E) return;
  const long stride = (long)prm.E * NFK;
  const int N = prm.N;
  // the element's nodes (face seeds) and its face records
  if (!in_bounds(prm.status, (long long)e * NP + NP - 1, N) || !in_bounds(prm.status, (long long)e * NFK + NFK - 1, stride))
    return;

  for (int t = a; t < NFK; t += NP) {
    const int f = t / NK, kk = t % NK;
    const int e2 = neighbour(prm, e, f);
    if (e2 >= 0 && (!in_bounds(prm.status, (long long)e2 * NP + NP - 1, N) ||
                    !in_bounds(prm.status, (long long)e2 * NFK + NFK - 1, stride)))
      continue;
    const bool wall = e2 < 0;
    const bool xf = f < 2;
    const double sg = (f & 1) ? 1.0 : -1.0;
    const double mx = xf ? sg : 0.0, my = xf ? 0.0 : sg;
    const double wf = xf ? wfx[kk] : wfy[kk];
    double Tm[NT], Tp[NT];
    const long om = (long)e * NFK + t;
#pragma unroll
    for (int q = 0; q < NT; ++q) Tm[q] = __ldg(tr + q * stride + om);
    int flip_u = 0, flip_v = 0;  // wall ghost sign flips
    if (!wall) {
      const long op = (long)e2 * NFK + (f ^ 1) * NK + kk;
#pragma unroll
      for (int q = 0; q < NT; ++q) Tp[q] = __ldg(tr + q * stride + op);
    } else {
#pragma unroll
      for (int q = 0; q < NT; ++q) Tp[q] = Tm[q];
      if (prm.bc[f] == BC_SLIP) {
        flip_u = xf;
        flip_v = !xf;
      } else {
        flip_u = flip_v = 1;
      }
      if (flip_u) { Tp[T_RU] = -Tm[T_RU]; Tp[T_U] = -Tm[T_U]; }
      if (flip_v) { Tp[T_RV] = -Tm[T_RV]; Tp[T_V] = -Tm[T_V]; }
    }

    // seeds: own evaluation and (interior faces) the neighbour's evaluation
    double sSo[NV], sLo[6], sSn[NV] = {0, 0, 0, 0, 0, 0, 0}, sLn[6] = {0, 0, 0, 0, 0, 0};
    face_seeds<P, DIM>(lam, N, e, f, kk, Dx, Dy, invM, sSo, sLo);
    if (!wall) face_seeds<P, DIM>(lam, N, e2, f ^ 1, kk, Dx, Dy, invM, sSn, sLn);

    double bm[NT], bp[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) bm[q] = bp[q] = 0.0;

    // forward quantities
    const double unm = Tm[T_U] * mx + Tm[T_V] * my;
    const double unp = Tp[T_U] * mx + Tp[T_V] * my;
    const double Lm = fabs(unm) + Tm[T_C], Lp = fabs(unp) + Tp[T_C];
    const bool own = Lm >= Lp;
    const double lam_ = own ? Lm : Lp;
    double blam = 0.0, bunm = 0.0, bunp = 0.0;

    // (a) Lax-Friedrichs part of the conservative equations, seed = own - neighbour
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int vv = M1 + c;
      const double g = sSo[vv] - sSn[vv];
      const double bF = -0.5 * wf * g;  // adjoint of Fm and of Fp
      blam += wf * 0.5 * (Tp[vv] - Tm[vv]) * g;
      bp[vv] += wf * lam_ * 0.5 * g;
      bm[vv] -= wf * lam_ * 0.5 * g;
      if (c < 4) {
        bm[vv] += bF * unm;
        bunm += bF * Tm[vv];
        bp[vv] += bF * unp;
        bunp += bF * Tp[vv];
        if (c == 2) { bm[T_P] += bF * mx; bp[T_P] += bF * mx; }
        if (c == 3) { bm[T_P] += bF * my; bp[T_P] += bF * my; }
      } else {
        bm[T_RE] += bF * unm;
        bm[T_P] += bF * unm;
        bunm += bF * (Tm[T_RE] + Tm[T_P]);
        bp[T_RE] += bF * unp;
        bp[T_P] += bF * unp;
        bunp += bF * (Tp[T_RE] + Tp[T_P]);
      }
    }
    // (b) transport of phi and psi seen from this element: wf (lambda - m.u-) [[q]]
    // (c) ... and from the neighbour: wf (lambda + m.u+) (q- - q+)/2
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int vv = r == 0 ? T_PHI : T_PSI;
      const double hj = 0.5 * (Tp[vv] - Tm[vv]);
      const double go = sSo[r == 0 ? PHI : PSI], gn = sSn[r == 0 ? PHI : PSI];
      blam += wf * hj * go;
      bunm -= wf * hj * go;
      bp[vv] += wf * (lam_ - unm) * 0.5 * go;
      bm[vv] -= wf * (lam_ - unm) * 0.5 * go;
      blam += wf * (-hj) * gn;
      bunp += wf * (-hj) * gn;
      bm[vv] += wf * (lam_ + unp) * 0.5 * gn;
      bp[vv] -= wf * (lam_ + unp) * 0.5 * gn;
    }
    // (d) SIP flux of a_1 and of every a_1-derived term (seed = own - neighbour)
    if (!wall) {
      const double eta = xf ? prm.eta_x : prm.eta_y;
      const double jump = Tp[T_PHI] - Tm[T_PHI];
      const double gn = 0.5 * (Tp[T_GPHI] + Tm[T_GPHI]) * sg;
      const double sp = Tp[T_PHI] * (1.0 - Tp[T_PHI]), sm = Tm[T_PHI] * (1.0 - Tm[T_PHI]);
      const double sharp = 0.5 * (sp * Tp[T_N] + sm * Tm[T_N]) * sg;
      const double ahat = prm.Gamma * (prm.eps * (gn + eta * jump) - sharp);
      const double km = 0.5 * (Tm[T_U] * Tm[T_U] + Tm[T_V] * Tm[T_V]);
      const double kp = 0.5 * (Tp[T_U] * Tp[T_U] + Tp[T_V] * Tp[T_V]);
      const double Cq[6] = {1.0, prm.rho01, -prm.rho02, prm.drho0 * 0.5 * (Tp[T_U] + Tm[T_U]),
                            prm.drho0 * 0.5 * (Tp[T_V] + Tm[T_V]),
                            0.5 * (Tp[T_B] + Tm[T_B]) + prm.drho0 * 0.5 * (kp + km)};
      const double sym = -wf * 0.5 * prm.Gamma * prm.eps * jump;
      const int slot[6] = {PHI, M1, M2, RU, RV, RE};
      double bahat = 0.0, bsym = 0.0, bC[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const double gS = sSo[slot[c]] - sSn[slot[c]];
        const double gL = sLo[c] - sLn[c];
        bahat += wf * Cq[c] * gS;
        bC[c] = wf * ahat * gS + sym * gL;
        bsym += Cq[c] * gL;
      }
      double bjump = -wf * 0.5 * prm.Gamma * prm.eps * bsym;
      const double bgn = prm.Gamma * prm.eps * bahat;
      bjump += prm.Gamma * prm.eps * eta * bahat;
      const double bsharp = -prm.Gamma * bahat;
      bp[T_GPHI] += 0.5 * sg * bgn;
      bm[T_GPHI] += 0.5 * sg * bgn;
      const double bsp = 0.5 * sg * Tp[T_N] * bsharp, bsm = 0.5 * sg * Tm[T_N] * bsharp;
      bp[T_N] += 0.5 * sg * sp * bsharp;
      bm[T_N] += 0.5 * sg * sm * bsharp;
      bp[T_PHI] += (1.0 - 2.0 * Tp[T_PHI]) * bsp + bjump;
      bm[T_PHI] += (1.0 - 2.0 * Tm[T_PHI]) * bsm - bjump;
      bp[T_U] += prm.drho0 * 0.5 * bC[3];
      bm[T_U] += prm.drho0 * 0.5 * bC[3];
      bp[T_V] += prm.drho0 * 0.5 * bC[4];
      bm[T_V] += prm.drho0 * 0.5 * bC[4];
      bp[T_B] += 0.5 * bC[5];
      bm[T_B] += 0.5 * bC[5];
      const double bk = prm.drho0 * 0.5 * bC[5];
      bp[T_U] += Tp[T_U] * bk;
      bp[T_V] += Tp[T_V] * bk;
      bm[T_U] += Tm[T_U] * bk;
      bm[T_V] += Tm[T_V] * bk;
    }
    // (e) lambda = max of the one-sided speeds
    if (own) {
      bunm += (unm > 0.0 ? 1.0 : (unm < 0.0 ? -1.0 : 0.0)) * blam;
      bm[T_C] += blam;
    } else {
      bunp += (unp > 0.0 ? 1.0 : (unp < 0.0 ? -1.0 : 0.0)) * blam;
      bp[T_C] += blam;
    }
    // (f) normal velocities
    bm[T_U] += mx * bunm;
    bm[T_V] += my * bunm;
    bp[T_U] += mx * bunp;
    bp[T_V] += my * bunp;
    // (g) a wall's ghost is a function of the own trace
    if (wall) {
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const bool neg = ((q == T_RU || q == T_U) && flip_u) || ((q == T_RV || q == T_V) && flip_v);
        bm[q] += neg ? -bp[q] : bp[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) trbar[q * stride + om] = bm[q];
  }
}

template <int P, int DIM>
__global__ void __launch_bounds__(Geom<P, DIM, false, false>::THREADS)
k_adj_volume(const Params prm, const double *__restrict__ w, const double *__restrict__ lam,
             const double *__restrict__ trbar, double *__restrict__ out, double ca, const double *__restrict__ xa,
             double cb, double cc, const double *__restrict__ yc, double cd, const double *__restrict__ zd) {
  using G = Geom<P, DIM, false, false>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int P11 = P1 * P1;
  __shared__ double s_op[4 * P11];
  __shared__ double s_f[6][EPB][NP];

  for (int t = threadIdx.x; t < 4 * P11; t += blockDim.x) s_op[t] = prm.ops[t];
  const double *Dx = s_op, *Dy = s_op + P11, *Dhx = s_op + 2 * P11, *Dhy = s_op + 3 * P11;

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blockIdx.x * EPB + le;
  const int N = prm.N;
  const bool act = lane && e < prm.E && in_bounds(prm.status, (long long)e * NP + a, N);
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const long n = (long)(act ? e : 0) * NP + a;

  // ---- forward recomputation (as k_volume)
  double q[NV], lm[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    q[v] = act ? __ldg(w + (long)v * N + n) : (v == M1 || v == M2 ? 1.0 : 0.0);
    lm[v] = act ? __ldg(lam + (long)v * N + n) : 0.0;
  }
  const double phi = q[PHI];
  const double rho = q[M1] + q[M2];
  const double ir = 1.0 / rho;
  const double u = q[RU] * ir;
  const double v = DIM == 2 ? q[RV] * ir : 0.0;
  double Cm, den;
  const double Pr = sg_pressure(prm, phi, rho, q[RU], DIM == 2 ? q[RV] : 0.0, q[RE], &Cm, &den);
  const double B = fma(Pr, prm.Bp, prm.dC);
  const double k = 0.5 * (u * u + v * v);
  if (lane) {
    s_f[0][le][a] = phi;
    s_f[1][le][a] = q[PSI];
  }
  __syncthreads();
  double gpx = 0.0, gpy = 0.0, gsx = 0.0, gsy = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const double dx = Dx[i * P1 + c];
    gpx = fma(dx, s_f[0][le][c + P1 * j], gpx);
    gsx = fma(dx, s_f[1][le][c + P1 * j], gsx);
    if (DIM == 2) {
      const double dy = Dy[j * P1 + c];
      gpy = fma(dy, s_f[0][le][i + P1 * c], gpy);
      gsy = fma(dy, s_f[1][le][i + P1 * c], gsy);
    }
  }
  const double g2 = gsx * gsx + gsy * gsy;
  double nx = 0.0, ny = 0.0, rn = 0.0;
  const bool has_n = g2 >= 1e-24;
  if (has_n) {
    rn = rsqrt(g2);
    nx = gsx * rn;
    ny = gsy * rn;
  }
  const double sphi = phi * (1.0 - phi);
  const double a1x = prm.Gamma * (prm.eps * gpx - sphi * nx);
  const double a1y = prm.Gamma * (prm.eps * gpy - sphi * ny);
  const double cE = prm.drho0 * k + B;

  // ---- reverse of the volume contraction: Fbar = Dhat^T lambda (per equation)
  __syncthreads();
  if (lane) {
    s_f[0][le][a] = lm[PHI];
#pragma unroll
    for (int c = 1; c < 6; ++c) s_f[c][le][a] = lm[c + 1];
  }
  __syncthreads();
  double bF[12];
#pragma unroll
  for (int eq = 0; eq < 6; ++eq) {
    double bx = 0.0, by = 0.0;
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      bx = fma(Dhx[c * P1 + i], s_f[eq][le][c + P1 * j], bx);
      if (DIM == 2) by = fma(Dhy[c * P1 + j], s_f[eq][le][i + P1 * c], by);
    }
    bF[2 * eq] = bx;
    bF[2 * eq + 1] = by;
  }

  // adjoints of the node quantities
  double bw[NV] = {0, 0, 0, 0, 0, 0, 0};
  double bu = 0.0, bv = 0.0, bP = 0.0, bB = 0.0, bk = 0.0, bc = 0.0, brho = 0.0;
  double bgpx = 0.0, bgpy = 0.0, bgsx = 0.0, bgsy = 0.0, bnx = 0.0, bny = 0.0, ba1x = 0.0, ba1y = 0.0;

  // non-conservative transport of phi and psi
  bgpx -= lm[PHI] * u;
  bgpy -= lm[PHI] * v;
  bgsx -= lm[PSI] * u;
  bgsy -= lm[PSI] * v;
  bu -= lm[PHI] * gpx + lm[PSI] * gsx;
  bv -= lm[PHI] * gpy + lm[PSI] * gsy;
  if (prm.gravity) {
    brho += lm[RU] * prm.gx + lm[RV] * prm.gy + lm[RE] * (prm.gx * u + prm.gy * v);
    bu += lm[RE] * rho * prm.gx;
    bv += lm[RE] * rho * prm.gy;
  }
  // face-trace adjoints of the faces this node lies on
  const bool onW = i == 0, onE = i == P, onS = DIM == 2 && j == 0, onN = DIM == 2 && j == P;
  if (act && (onW || onE || onS || onN)) {
    const long stride = (long)prm.E * NFK;
    auto take = [&](int f, int kk, bool xaxis) {
      const long o = (long)e * NFK + f * NK + kk;
      if (!in_bounds(prm.status, o, stride)) return;
      double T[NT_INVISCID];
#pragma unroll
      for (int qf = 0; qf < NT_INVISCID; ++qf) T[qf] = __ldg(trbar + qf * stride + o);
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) bw[vv] += T[vv];
      bu += T[T_U];
      bv += T[T_V];
      bP += T[T_P];
      bc += T[T_C];
      bB += T[T_B];
      if (xaxis) { bgpx += T[T_GPHI]; bnx += T[T_N]; }
      else       { bgpy += T[T_GPHI]; bny += T[T_N]; }
    };
    const int kx = DIM == 2 ? j : 0;
    if (onW) take(0, kx, true);
    if (onE) take(1, kx, true);
    if (onS) take(2, i, false);
    if (onN) take(3, i, false);
  }
  // fluxes
  ba1x -= bF[0];
  ba1y -= bF[1];
  bw[M1] += bF[2] * u + bF[3] * v;
  bu += bF[2] * q[M1];
  bv += bF[3] * q[M1];
  ba1x -= prm.rho01 * bF[2];
  ba1y -= prm.rho01 * bF[3];
  bw[M2] += bF[4] * u + bF[5] * v;
  bu += bF[4] * q[M2];
  bv += bF[5] * q[M2];
  ba1x += prm.rho02 * bF[4];
  ba1y += prm.rho02 * bF[5];
  // F6 = ru u + P - drho0 a1x u ; F7 = ru v - drho0 a1y u
  bw[RU] += bF[6] * u + bF[7] * v;
  bu += bF[6] * (q[RU] - prm.drho0 * a1x) - prm.drho0 * a1y * bF[7];
  bv += bF[7] * q[RU];
  bP += bF[6];
  ba1x -= prm.drho0 * u * bF[6];
  ba1y -= prm.drho0 * u * bF[7];
  // F8 = rv u - drho0 a1x v ; F9 = rv v + P - drho0 a1y v
  bw[RV] += bF[8] * u + bF[9] * v;
  bu += bF[8] * q[RV];
  bv += bF[9] * (q[RV] - prm.drho0 * a1y) - prm.drho0 * a1x * bF[8];
  bP += bF[9];
  ba1x -= prm.drho0 * v * bF[8];
  ba1y -= prm.drho0 * v * bF[9];
  // F10 = (rE + P) u - cE a1x ; F11 = (rE + P) v - cE a1y
  bw[RE] += bF[10] * u + bF[11] * v;
  bP += bF[10] * u + bF[11] * v;
  bu += bF[10] * (q[RE] + Pr);
  bv += bF[11] * (q[RE] + Pr);
  const double bcE = -(bF[10] * a1x + bF[11] * a1y);
  ba1x -= cE * bF[10];
  ba1y -= cE * bF[11];
  bk += prm.drho0 * bcE;
  bB += bcE;
  // a_1 = Gamma (eps grad phi - phi (1 - phi) n)
  bgpx += prm.Gamma * prm.eps * ba1x;
  bgpy += prm.Gamma * prm.eps * ba1y;
  const double bs = -prm.Gamma * (nx * ba1x + ny * ba1y);
  bnx -= prm.Gamma * sphi * ba1x;
  bny -= prm.Gamma * sphi * ba1y;
  bw[PHI] += (1.0 - 2.0 * phi) * bs;
  // n = grad psi / |grad psi|
  if (has_n) {
    const double nn = nx * bnx + ny * bny;
    bgsx += rn * (bnx - nx * nn);
    bgsy += rn * (bny - ny * nn);
  }
  // reverse of the gradient contractions (transpose over the element)
  __syncthreads();
  if (lane) {
    s_f[0][le][a] = bgpx;
    s_f[1][le][a] = bgpy;
    s_f[2][le][a] = bgsx;
    s_f[3][le][a] = bgsy;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const double dx = Dx[c * P1 + i];
    bw[PHI] = fma(dx, s_f[0][le][c + P1 * j], bw[PHI]);
    bw[PSI] = fma(dx, s_f[2][le][c + P1 * j], bw[PSI]);
    if (DIM == 2) {
      const double dy = Dy[c * P1 + j];
      bw[PHI] = fma(dy, s_f[1][le][i + P1 * c], bw[PHI]);
      bw[PSI] = fma(dy, s_f[3][le][i + P1 * c], bw[PSI]);
    }
  }
  // closure: c (face nodes), k, B, P, u, v, rho
  // (one reciprocal of the mixture denominator: this kernel is bound by the FP64 pipe, where each
  // division is several operations)
  double bCm = 0.0, bden = 0.0, bir = 0.0;
  const double iden = 1.0 / den;
  if (bc != 0.0) {
    const double PC = Pr + Cm;
    const double X = Pr + PC * iden;
    const double c = sqrt(X * ir);
    const double h = 0.5 / c;  // 1 / (2 c)
    const double bX = bc * ir * h;
    bir += bc * X * h;
    bP += bX * (1.0 + iden);
    bCm += bX * iden;
    bden -= bX * PC * iden * iden;
  }
  bu += u * bk;
  bv += v * bk;
  bP += prm.Bp * bB;
  // P = (rhoE - rhok - Cm) / den, rhok = (ru^2 + rv^2) / (2 rho)
  const double bPd = bP * iden;
  const double brhoe = bPd;
  bCm -= bPd;
  bden -= bPd * Pr;
  bw[RE] += brhoe;
  const double brhok = -brhoe;
  bw[RU] += brhok * q[RU] * ir;
  if (DIM == 2) bw[RV] += brhok * q[RV] * ir;
  brho -= brhok * 0.5 * (q[RU] * q[RU] + (DIM == 2 ? q[RV] * q[RV] : 0.0)) * ir * ir;
  bw[PHI] += (prm.C1 - prm.C2) * bCm + (prm.g1 - prm.g2) * bden;
  bw[RU] += bu * ir;
  bir += bu * q[RU];
  if (DIM == 2) {
    bw[RV] += bv * ir;
    bir += bv * q[RV];
  }
  brho -= bir * ir * ir;
  bw[M1] += brho;
  bw[M2] += brho;

  if (!act) return;
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) {
    const long o = (long)vv * N + n;
    double r = cb * bw[vv];
    if (xa) r = fma(ca, __ldg(xa + o), r);
    if (yc) r = fma(cc, __ldg(yc + o), r);
    if (zd) r = fma(cd, __ldg(zd + o), r);
    out[o] = r;
  }
}

struct AdjKernels {
  cudaError_t (*face)(const Params &, const double *lam, const double *trace, double *trbar, cudaStream_t);
  cudaError_t (*volume)(const Params &, const double *w, const double *lam, const double *trbar, double *out,
                        double ca, const double *xa, double cb, double cc, const double *yc, double cd,
                        const double *zd, cudaStream_t);
};

template <int P, int DIM>
cudaError_t launch_adj_face(const Params &prm, const double *lam, const double *trace, double *trbar,
                            cudaStream_t s) {
  using G = Geom<P, DIM, false, false>;
  k_adj_face<P, DIM><<<(prm.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(prm, lam, trace, trbar);
  return cudaGetLastError();
}

template <int P, int DIM>
cudaError_t launch_adj_volume(const Params &prm, const double *w, const double *lam, const double *trbar,
                              double *out, double ca, const double *xa, double cb, double cc, const double *yc,
                              double cd, const double *zd, cudaStream_t s) {
  using G = Geom<P, DIM, false, false>;
  k_adj_volume<P, DIM><<<(prm.E + G::EPB - 1) / G::EPB, G::THREADS, 0, s>>>(prm, w, lam, trbar, out, ca, xa, cb,
                                                                           cc, yc, cd, zd);
  return cudaGetLastError();
}

template <int P>
bool adj_kernels_p(int dim, AdjKernels *out) {
  if (dim == 1) *out = {&launch_adj_face<P, 1>, &launch_adj_volume<P, 1>};
  else *out = {&launch_adj_face<P, 2>, &launch_adj_volume<P, 2>};
  return true;
}

bool adj_kernels(int p, int dim, AdjKernels *out);

}  // namespace dgpf
