// dg_kernels_fp32.cuh -- FP32-bulk kernels of the DG right-hand side (GB300, sm_103a).
//
// GB300 executes FP64 at about 1/73 of its FP32 rate, so this path keeps FP64
// out of the stage loop.  Internally the state is held in FP32 with the total
// energy replaced by the reduced energy
//     rhoEt = rho E - Cmix(phi),   Cmix(phi) = C_2 + (C_1 - C_2) phi,
//     C_l = gamma_l Pinf_l / (gamma_l - 1),
// i.e. rho E minus the stiffened-gas constant of Sec. 2.  The pressure is then
// P = (rhoEt - rho k) / (phi g_1 + (1 - phi) g_2) with no cancellation, so it
// is accurate in FP32.  The FP64 pressure recovery happens once per dg_step
// call, in the conversion kernels (k_to32 / k_to64).
//
// Evolution of rhoEt.  With the collocated GLL quadrature the weak-form volume
// term satisfies summation by parts, and the right-hand side of rhoEt,
// L(rhoEt) = L(rho E) - (C_1 - C_2) L(phi), equals -- exactly, in exact
// arithmetic -- the energy equation of the paper with rhoEt in place of rho E
// in the convective flux, B - (C_1 - C_2) = P (gamma_1 g_1 - gamma_2 g_2) as
// the a_1 coefficient, and a compression term
//     - sum_c D_ic Cmix(phi_c) (u_c - u_i)              (volume, per direction)
//     - M^-1 int l_i 1/2 Cmix(phi+) (u+ - u-) . m       (faces).
// Written with velocity differences, this term vanishes to rounding in a
// uniform flow, which is what keeps the pressure at interfaces in FP32.
// All other terms are those of the FP64 kernels (dg_kernels_fp64.cuh), but
// written in the strong form, which summation by parts makes identical to the
// weak form of Sec. 3:  L_i = -(div_h F)_i + M^-1 int l_i (F- - F^) . m.
// Every derivative is contracted over differences, sum_c D_ic (f_c - f_i)
// (D annihilates constants), and every face term is a difference F- - F^.
// In FP32 this makes the rounding error scale with the variation of a field
// rather than with its offset (P ~ 1e5, psi, phi ~ 1), and keeps a uniform
// state exactly steady.
//
// Accumulation.  The step start is carried as a float-float pair (hi, lo),
// hi + lo holding ~48 significant bits, and the three SSP-RK3 stages as FP32
// increments over it (Shu-Osher form rewritten for the increments):
//     d1 = dt L(w0),  d2 = (d1 + dt L(w0 + d1)) / 4,  d3 = 2 (d2 + dt L(w0 + d2)) / 3,
//     w_{n+1} = w0 + d3,
// where each right-hand side is evaluated on the FP32 state hi + d (rounded).
// The increments are small next to the state (the acoustic time step moves a
// field by a few parts in 1e5 per step), so they keep FP32's relative precision
// of the change, and w0 + d3 is added in float-float (two-sum): the state does
// not lose the low bits of each step's change to FP32 rounding, which over
// thousands of steps otherwise grows to ~1e-5 of the field.
//
// The first stage of a step can read the FP64 state directly (splitting it into
// hi and lo on load and writing the FP32 internal state), and the last stage
// can write the FP64 state directly (hi + lo).  With the fused stage kernel
// (k_surfvol32 below) n steps take 1 + 3n launches.
#pragma once

#include "dg_common.cuh"
#include "dg_kernels_fp64.cuh"
#include "dg_pdl.cuh"

namespace dgpf {

// Single-precision copy of the closure constants.
struct ParamsF {
  float C2, dC, g1, g2, Bp;
  float rho01, rho02, drho0, mu1, mu2, sigma, gx, gy, Gamma, eps, eta_x, eta_y;
};

__host__ inline ParamsF to_float(const Params &p) {
  return ParamsF{(float)p.C2, (float)p.dC, (float)p.g1, (float)p.g2, (float)p.Bp, (float)p.rho01, (float)p.rho02,
                 (float)p.drho0, (float)p.mu1, (float)p.mu2, (float)p.sigma, (float)p.gx, (float)p.gy,
                 (float)p.Gamma, (float)p.eps, (float)p.eta_x, (float)p.eta_y};
}

// Face-trace record of the FP32-bulk kernels: the seven state values (in the
// order of Var) and what needs the whole element -- d(phi)/d(axis normal to
// the face), the level-set normal component on that axis and, viscous, the
// stress components tau . e_axis.  Viscous kernels: velocity, pressure, sound
// speed, B and the mixture viscosity are recomputed from the state by the
// reader (trace_derive).  Inviscid kernels: pressure, sound speed and 1/rho
// travel in the record's spare words (C_P, C_C, C_IR) and the reader only
// multiplies (trace_stored).  (Viscous records of 64 bytes carrying P, c and
// 1/rho as well were measured slower at 256x256 p4: the kernels are close
// enough to the memory bound that the extra 16 bytes per record cost more than
// the closure they save.)
enum TraceField32 { C_GPHI = 7, C_N = 8, C_TX = 9, C_TY = 10 };
constexpr int NT32_INVISCID = 9;
constexpr int NT32_VISCOUS = 11;
// The FP32 face traces are stored one 48-byte record per face node ([E * NFK][TRW32] floats, the
// words in TraceField32 order, the rest padding), so that a record moves in three 128-bit
// accesses instead of nine or eleven scalar ones.
constexpr int TRW32 = 12;
enum TraceClosure32 { C_P = 9, C_C = 10, C_IR = 11 };
// The FP32 internal state and volume parts of the inviscid kernels are stored one 32-byte record
// per node ([N][SW32] floats: the seven variables and a padding word), moved in two 128-bit
// accesses; the viscous kernels keep them field-major ([7][N]), where the records did not pay
// (256x256 p4 Rayleigh-Taylor step 0.301 -> 0.316 ms), while the inviscid batch gained 11%.
constexpr int SW32 = 8;

// Loads of data that an earlier kernel wrote: non-coherent (__ldg) in a kernel
// launched plainly, coherent (__ldca) in one launched as a programmatic
// dependent (COH), which overlaps the kernel that writes the data.
template <bool COH, typename T>
__device__ __forceinline__ T ld_in(const T *p) {
  if (COH) return __ldca(p);
  return __ldg(p);
}

template <bool AOS, bool COH = false>
__device__ __forceinline__ void load_node32(const float *__restrict__ w, long n, int N, float *q) {
  if (AOS) {
    const float4 *r = reinterpret_cast<const float4 *>(w) + 2 * n;
    const float4 a = ld_in<COH>(r), b = ld_in<COH>(r + 1);
    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
    q[4] = b.x; q[5] = b.y; q[6] = b.z;
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = ld_in<COH>(w + (long)v * N + n);
  }
}

template <bool AOS>
__device__ __forceinline__ void store_node32(float *w, long n, int N, const float *q) {
  if (AOS) {
    float4 *r = reinterpret_cast<float4 *>(w) + 2 * n;
    r[0] = make_float4(q[0], q[1], q[2], q[3]);
    r[1] = make_float4(q[4], q[5], q[6], 0.f);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) w[(long)v * N + n] = q[v];
  }
}

// Buffers of one stage kernel (each a node-record or field-major FP32 array like
// the internal state, except out64 and w64in): the step start hi part w0 (all
// stage modes) and lo part lo (MODE_S3), the previous stage's increment din
// (MODE_S2, MODE_S3), this stage's increment dout (MODE_S1, MODE_S2), the new
// step start hi_out / lo_out (MODE_S3 when the step is not the last of the
// call), and the FP64 output out64 (MODE_RHS: L; MODE_S3 at the end of a call:
// the state).  w64in (MODE_S3 with out64, when the step start is the FP64 state
// itself, i.e. the call's only step): the last increment is added to it in FP64
// (in place when w64in == out64), and w0 and lo are not read.
struct StageIO {
  const float *w0, *lo, *din;
  float *dout, *hi_out, *lo_out;
  double *out64;
  const double *w64in;
  const double *dt_dev;  // step size read at run time (captured step sequences), else NULL
};

// (hi, lo) + d in float-float arithmetic: Knuth's two-sum of hi and d, the
// error added to lo, then a fast two-sum to renormalise (|s| >= |t|).  The
// intrinsics keep every operation separately rounded (no contraction).
__device__ __forceinline__ void ff_add(float &hi, float &lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float t = __fadd_rn(lo, err);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// FP64 <-> float-float conversions at the ends of a call, by integer operations
// on the bit patterns.  On GB300 every conversion instruction (F2F, I2F) and
// every FP64 add runs on the reduced FP64 pipe, where the split and the sum of
// seven variables per node cost more than the kernel's FP32 work.

// An integer k in [0, 2^23) as a float, exactly (the float 2^23 + k minus 2^23).
__device__ __forceinline__ float small_int_to_float(unsigned k) {
  return __uint_as_float(0x4B000000u | k) - 8388608.0f;
}

// Split an FP64 value into floats hi + lo: hi is the value rounded to 24
// significant bits (ties away from zero; the top 24 bits of the significand
// plus one unit when the dropped 29 bits reach half a unit), lo the remainder
// (the dropped bits less that unit, in units of the double's last place)
// rounded once to 24 bits.  Magnitudes below 2^-74 split into zeros (lo would
// be below the normal floats); 2^126 and above, infinities and NaNs give an
// infinity or a NaN in hi (the state is then non-physical and is flagged).
__device__ __forceinline__ void split_ff(double d, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned e = (hw >> 20) & 0x7FFu, sign = hw & 0x80000000u;
  if (e < 949u) {
    hi = lo = __uint_as_float(sign);
    return;
  }
  if (e > 1148u) {
    const bool nan = e == 0x7FFu && ((hw & 0xFFFFFu) | lw);
    hi = __uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
    lo = 0.f;
    return;
  }
  const unsigned low29 = lw & 0x1FFFFFFFu;
  const bool up = low29 >= 0x10000000u;
  const unsigned long long bh = (b & ~0x1FFFFFFFull) + (up ? 0x20000000ull : 0ull);
  const unsigned hhw = (unsigned)(bh >> 32), hlw = (unsigned)bh;
  const unsigned he = (hhw >> 20) & 0x7FFu;
  hi = __uint_as_float(sign | ((he - 896u) << 23) | ((hhw & 0xFFFFFu) << 3) | (hlw >> 29));
  // |remainder| in units of 2^(e - 1075), below 2^28: two exact pieces, one rounding
  const unsigned m = up ? 0x20000000u - low29 : low29;
  const float mag = fmaf(small_int_to_float(m >> 14), 16384.0f, small_int_to_float(m & 0x3FFFu));
  const float unit = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075), a normal float
  lo = __uint_as_float(__float_as_uint(mag * unit) ^ ((sign != 0u) != up ? 0x80000000u : 0u));
}

// The FP64 value of the float pair hi + lo (|lo| at most one unit of hi's last
// place, as ff_add leaves it): the two significands aligned in units of 2^-29
// of hi's last place, added or subtracted as integers, renormalised and packed
// (bits of lo below the double's last place are dropped).  lo zero or below
// the normal floats contributes nothing; hi zero, subnormal, infinite or NaN
// is converted on its own (subnormals to zero).
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
  const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const unsigned eh = (uh >> 23) & 0xFFu, el = (ul >> 23) & 0xFFu, sign = uh & 0x80000000u;
  if (eh == 0u) return __hiloint2double((int)sign, 0);
  if (eh == 0xFFu) return __hiloint2double((int)(sign | 0x7FF00000u | ((uh & 0x7FFFFFu) ? 0x80000u : 0u)), 0);
  const unsigned long long H = (unsigned long long)(0x800000u | (uh & 0x7FFFFFu)) << 29;
  const int s = (int)el - (int)eh + 29;
  unsigned long long L = 0ull;
  if (el != 0u && s > -24) {
    const unsigned Ml = 0x800000u | (ul & 0x7FFFFFu);
    L = s >= 0 ? (unsigned long long)Ml << s : (unsigned long long)(Ml >> (-s));
  }
  unsigned long long M = ((ul ^ uh) & 0x80000000u) ? H - L : H + L;
  int E = (int)eh;
  if (M >= (1ull << 53)) {
    M >>= 1;
    ++E;
  } else if (M < (1ull << 52)) {
    M <<= 1;
    --E;
  }
  const unsigned long long bits = ((unsigned long long)sign << 32) | ((unsigned long long)(E + 896) << 52) |
                                  (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Exact float -> double by the same bit manipulation (subnormals to zero).
__device__ __forceinline__ double f2d(float f) { return ff_to_double(f, 0.f); }

// The closure's divisions (by rho and by the mixture 1/(gamma-1)) use the
// approximate reciprocal (__fdividef: within 2 ulp for the magnitudes of a
// density or of 1/(gamma-1)), far below the FP32 storage error of this path;
// the IEEE division costs about four times the instructions.
__device__ __forceinline__ float rcp32(float x) { return __fdividef(1.0f, x); }

// Fill T[T_U], T[T_V], T[T_P], T[T_C], T[T_B] (and T[T_MU]) from the state
// values T[T_PHI..T_RE], with the operations of the volume body.
template <int DIM, bool VISC>
__device__ __forceinline__ void trace_derive(const ParamsF &pf, float *T) {
  const float phi = T[T_PHI];
  const float rho = T[T_M1] + T[T_M2];
  const float ir = rcp32(rho);
  const float u = T[T_RU] * ir;
  const float v = DIM == 2 ? T[T_RV] * ir : 0.f;
  const float k = 0.5f * (u * u + v * v);
  const float iG = rcp32(fmaf(phi, pf.g1 - pf.g2, pf.g2));
  const float Pr = (T[T_RE] - rho * k) * iG;
  const float Cm = fmaf(pf.dC, phi, pf.C2);
  T[T_U] = u;
  T[T_V] = v;
  T[T_P] = Pr;
  T[T_C] = sqrtf((Pr + (Pr + Cm) * iG) * ir);
  T[T_B] = Pr * pf.Bp;
  if (VISC) T[T_MU] = pf.mu1 * phi + pf.mu2 * (1.f - phi);
}

// The inviscid reader's counterpart of trace_derive: velocity from the stored 1/rho, pressure and
// sound speed as stored by the writer, B from the pressure.
template <int DIM>
__device__ __forceinline__ void trace_stored(const ParamsF &pf, const float *C, float *T) {
  const float ir = C[C_IR];
  T[T_U] = T[T_RU] * ir;
  T[T_V] = DIM == 2 ? T[T_RV] * ir : 0.f;
  T[T_P] = C[C_P];
  T[T_C] = C[C_C];
  T[T_B] = C[C_P] * pf.Bp;
}

// Element lines in shared memory.  Every field a contraction reads is stored
// per element by rows (the x-lines, i fastest) and, for the y-derivatives, by
// columns (the y-lines, j fastest), so that a thread reads a whole line in the
// widest aligned loads the line length allows (P + 1 = 4: one 128-bit load;
// P + 1 = 2 or 6: 64-bit loads; odd lengths: one load per node) instead of one
// load per node.  (Padding odd lines to 16 bytes was measured slower at
// p = 4: the padded stride makes shared-memory bank conflicts.)
template <int P1>
__device__ __forceinline__ void load_line(const float *row, float *v) {
  if (P1 % 4 == 0) {
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int k = 0; k < P1 / 4; ++k) {
      const float4 x = r4[k];
      v[4 * k] = x.x;
      v[4 * k + 1] = x.y;
      v[4 * k + 2] = x.z;
      v[4 * k + 3] = x.w;
    }
  } else if (P1 % 2 == 0) {
    const float2 *r2 = reinterpret_cast<const float2 *>(row);
#pragma unroll
    for (int k = 0; k < P1 / 2; ++k) {
      const float2 x = r2[k];
      v[2 * k] = x.x;
      v[2 * k + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < P1; ++k) v[k] = row[k];
  }
}

// Volume kernel body for the element tile `blk` (EPB elements) of one problem.
// opsf: FP32 operator table (OpsLayout).  w64 != NULL: read the FP64 state and
// write the FP32 internal state to w32out (first stage of a step), and, when
// w64copy != NULL, the FP64 values as read into w64copy.  qin !=
// NULL: the thread's node state is already in registers (fused kernel).
// s_op: the block's shared copy of the operator table; this body copies the
// two derivative matrices into it unless ops_ready (the fused kernel's
// surface part has copied the whole table and synchronised the block).
template <int P, int DIM, bool VISC, bool ST, int EPBX = 0, bool PDL = false>
__device__ __forceinline__ void vol32_body(const Params &prm, const ParamsF &pf, const float *__restrict__ opsf,
                                           float *s_op, bool ops_ready, int blk, const float *__restrict__ w,
                                           float *__restrict__ rvol, float *__restrict__ tr,
                                           const double *__restrict__ w64, float *__restrict__ w32out,
                                           const float *qin = nullptr, float *__restrict__ lo_out = nullptr,
                                           double *__restrict__ w64copy = nullptr) {
  using G = Geom<P, DIM, VISC, ST, EPBX>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int P11 = P1 * P1;
  constexpr int NS = 12;
  constexpr int LS = P1;
  constexpr int NLY = DIM == 2 ? P1 : 1;  // lines per element in each orientation
  // Even line lengths: y-lines from a column copy in vector loads, the node's rows of D held in
  // registers.  Odd ones: y-lines read across the rows one node at a time and D read where used,
  // which the register-capped viscous kernels need (p = 4: the column copies and held rows cost 7%).
  constexpr bool COLS = DIM == 2 && P1 % 2 == 0;
  // rows (x-lines) of six fields per element and, when COLS, their columns (y-lines); without COLS
  // the y-flux components take six more row slots
  __shared__ __align__(16) float s_row[COLS || DIM == 1 ? 6 : 12][EPB][NLY][LS];
  __shared__ __align__(16) float s_col[COLS ? 6 : 1][EPB][COLS ? P1 : 1][LS];

  if (!ops_ready)
    for (int t = threadIdx.x; t < 2 * P11; t += blockDim.x) s_op[t] = opsf[t];
  const float *Dx = s_op, *Dy = s_op + P11;

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blk * EPB + le;
  const int N = prm.N;
  const bool act = lane && e < prm.E && in_bounds(prm.status, (long long)e * NP + a, N);
  const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
  const long n = (long)(act ? e : 0) * NP + a;

  float q[NV];
  if (qin) {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = act ? qin[v] : (v == M1 || v == M2 ? 1.f : 0.f);
  } else if (w64) {
    // first stage: split the FP64 state into hi + lo (the stiffened-gas constant leaves rho E
    // in FP64 first)
    double d[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) d[v] = act ? ld_in<PDL>(w64 + (long)v * N + n) : (v == M1 || v == M2 ? 1.0 : 0.0);
    if (w64copy && act) {
      // a device copy of a state in host memory, for the last stage to add to (one read over the
      // host link per call instead of two)
#pragma unroll
      for (int v = 0; v < NV; ++v) w64copy[(long)v * N + n] = d[v];
    }
    d[RE] = d[RE] - fma(prm.dC, d[PHI], prm.C2);
    if (lo_out) {
      // a call of several steps carries the step start as hi + lo
      float lo[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) split_ff(d[v], q[v], lo[v]);
      if (act) store_node32<!VISC>(lo_out, n, N, lo);
    } else {
      // a single step adds its last increment to the FP64 state itself: hi alone
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = __double2float_rn(d[v]);
    }
    if (act) store_node32<!VISC>(w32out, n, N, q);
  } else if (act) {
    load_node32<!VISC, PDL>(w, n, N, q);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = v == M1 || v == M2 ? 1.f : 0.f;
  }
  const float phi = q[PHI], psi = q[PSI];
  const float rho = q[M1] + q[M2];
  const float ir = rcp32(rho);
  const float u = q[RU] * ir;
  const float v = DIM == 2 ? q[RV] * ir : 0.f;
  const float k = 0.5f * (u * u + v * v);
  const float iG = rcp32(fmaf(phi, pf.g1 - pf.g2, pf.g2));
  const float Pr = (q[RE] - rho * k) * iG;
  const float Bq = Pr * pf.Bp;  // B - (C_1 - C_2)
  // Non-physical state: rho <= 0, a mixture 1/(gamma - 1) <= 0, or P + Pinf_mix <= 0, i.e.
  // rho c^2 = P + (P + Cm) / den <= 0 (Sec. 2 mixture rules).
  if (prm.check_finite && act && (rho <= 0.f || iG <= 0.f || Pr + (Pr + fmaf(pf.dC, phi, pf.C2)) * iG <= 0.f))
    atomicOr(prm.status, STATUS_NONPHYSICAL);

  if (lane) {
    s_row[0][le][j][i] = phi;
    s_row[1][le][j][i] = psi;
    s_row[2][le][j][i] = u;
    if (VISC) s_row[3][le][j][i] = v;
    if (COLS) {
      s_col[0][le][i][j] = phi;
      s_col[1][le][i][j] = psi;
      s_col[3][le][i][j] = v;
      if (VISC) s_col[2][le][i][j] = u;
    } else if (DIM == 2) {
      s_row[3][le][j][i] = v;
    }
  }
  __syncthreads();  // also orders the operator table's copy (above, or in the caller) before its reads
  // the node's rows of the two derivative matrices (held in registers when COLS)
  float dxr[P1], dyr[P1];
  if (COLS) {
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      dxr[c] = Dx[i * P1 + c];
      dyr[c] = Dy[j * P1 + c];
    }
  }
  auto DX = [&](int c) { return COLS ? dxr[c] : Dx[i * P1 + c]; };
  auto DY = [&](int c) { return COLS ? dyr[c] : Dy[j * P1 + c]; };
  auto s_fy = [&](int eq) -> float * { return &s_row[COLS || DIM == 1 ? 0 : 6 + eq][le][0][0]; };
  // the y-line of field slot f through the node
  auto yline = [&](int f, float *lv) {
    if (COLS) {
      load_line<P1>(&s_col[f][le][i][0], lv);
    } else {
#pragma unroll
      for (int c = 0; c < P1; ++c) lv[c] = s_row[f][le][c][i];
    }
  };

  float gpx = 0.f, gpy = 0.f, gsx = 0.f, gsy = 0.f, gux = 0.f, guy = 0.f, gvx = 0.f, gvy = 0.f, comp = 0.f;
  {
    float lp[P1], lq[P1];
    load_line<P1>(&s_row[0][le][j][0], lp);  // phi along x
    load_line<P1>(&s_row[2][le][j][0], lq);  // u along x
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      gpx = fmaf(DX(c), lp[c] - phi, gpx);
      comp = fmaf(DX(c) * fmaf(pf.dC, lp[c], pf.C2), lq[c] - u, comp);
      if (VISC) gux = fmaf(DX(c), lq[c] - u, gux);
    }
    load_line<P1>(&s_row[1][le][j][0], lp);  // psi along x
#pragma unroll
    for (int c = 0; c < P1; ++c) gsx = fmaf(DX(c), lp[c] - psi, gsx);
    if (VISC) {
      load_line<P1>(&s_row[3][le][j][0], lp);  // v along x
#pragma unroll
      for (int c = 0; c < P1; ++c) gvx = fmaf(DX(c), lp[c] - v, gvx);
    }
    if (DIM == 2) {
      yline(0, lp);  // phi along y
      yline(3, lq);  // v along y
#pragma unroll
      for (int c = 0; c < P1; ++c) {
        gpy = fmaf(DY(c), lp[c] - phi, gpy);
        comp = fmaf(DY(c) * fmaf(pf.dC, lp[c], pf.C2), lq[c] - v, comp);
        if (VISC) gvy = fmaf(DY(c), lq[c] - v, gvy);
      }
      yline(1, lp);  // psi along y
#pragma unroll
      for (int c = 0; c < P1; ++c) gsy = fmaf(DY(c), lp[c] - psi, gsy);
      if (VISC) {
        yline(2, lp);  // u along y
#pragma unroll
        for (int c = 0; c < P1; ++c) guy = fmaf(DY(c), lp[c] - u, guy);
      }
    }
  }

  // n = 0 where |grad psi| cannot be told from zero: FP32 storage of a
  // distance-like psi leaves ~1e-6 of noise in its gradient (the FP64 path
  // uses 1e-12), so below 1e-4 the direction is noise.
  const float g2 = gsx * gsx + gsy * gsy;
  float nx = 0.f, ny = 0.f;
  if (g2 >= 1e-8f) {
    const float r = rsqrtf(g2);
    nx = gsx * r;
    ny = gsy * r;
  }
  const float sphi = phi * (1.f - phi);
  const float a1x = pf.Gamma * (pf.eps * gpx - sphi * nx);
  const float a1y = pf.Gamma * (pf.eps * gpy - sphi * ny);

  float txx = 0.f, txy = 0.f, tyy = 0.f, mu = 0.f;
  if (VISC) {
    mu = pf.mu1 * phi + pf.mu2 * (1.f - phi);
    const float div3 = (gux + gvy) * (1.f / 3.f);
    txx = 2.f * mu * (gux - div3);
    tyy = 2.f * mu * (gvy - div3);
    txy = mu * (guy + gvx);
  }

  float kappa = 0.f;
  if (ST) {
    if (lane) {
      s_row[4][le][j][i] = nx;
      if (COLS) s_col[4][le][i][j] = ny;
      else if (DIM == 2) s_row[5][le][j][i] = ny;
    }
    __syncthreads();
    float dv = 0.f, lp[P1];
    load_line<P1>(&s_row[4][le][j][0], lp);
#pragma unroll
    for (int c = 0; c < P1; ++c) dv = fmaf(DX(c), lp[c] - nx, dv);
    if (DIM == 2) {
      yline(COLS ? 4 : 5, lp);
#pragma unroll
      for (int c = 0; c < P1; ++c) dv = fmaf(DY(c), lp[c] - ny, dv);
    }
    kappa = -dv;
  }

  const float cE = pf.drho0 * k + Bq;
  float F[NS];
  F[0] = -a1x;
  F[1] = -a1y;
  F[2] = q[M1] * u - pf.rho01 * a1x;
  F[3] = q[M1] * v - pf.rho01 * a1y;
  F[4] = q[M2] * u + pf.rho02 * a1x;
  F[5] = q[M2] * v + pf.rho02 * a1y;
  F[6] = q[RU] * u + Pr - pf.drho0 * a1x * u - txx;
  F[7] = q[RU] * v - pf.drho0 * a1y * u - txy;
  F[8] = q[RV] * u - pf.drho0 * a1x * v - txy;
  F[9] = q[RV] * v + Pr - pf.drho0 * a1y * v - tyy;
  F[10] = (q[RE] + Pr) * u - cE * a1x - (txx * u + txy * v);
  F[11] = (q[RE] + Pr) * v - cE * a1y - (txy * u + tyy * v);
  __syncthreads();
  // (odd line lengths: the y-components in slots 6..11 of the row layout, s_row and s_col being
  // one array there -- see below)
  if (lane) {
#pragma unroll
    for (int eq = 0; eq < 6; ++eq) {
      s_row[eq][le][j][i] = F[2 * eq];
      if (COLS) s_col[eq][le][i][j] = F[2 * eq + 1];
      else if (DIM == 2) s_fy(eq)[j * P1 + i] = F[2 * eq + 1];
    }
  }
  __syncthreads();

  // Strong-form volume term -(div_h F)_i, contracted over differences.
  float R[NV];
#pragma unroll
  for (int eq = 0; eq < 6; ++eq) {
    float acc = 0.f, lp[P1];
    const float fx = F[2 * eq], fy = F[2 * eq + 1];
    load_line<P1>(&s_row[eq][le][j][0], lp);
#pragma unroll
    for (int c = 0; c < P1; ++c) acc = fmaf(DX(c), lp[c] - fx, acc);
    if (COLS) {
      load_line<P1>(&s_col[eq][le][i][0], lp);
#pragma unroll
      for (int c = 0; c < P1; ++c) acc = fmaf(DY(c), lp[c] - fy, acc);
    } else if (DIM == 2) {
#pragma unroll
      for (int c = 0; c < P1; ++c) acc = fmaf(DY(c), s_fy(eq)[c * P1 + i] - fy, acc);
    }
    R[eq == 0 ? PHI : eq + 1] = -acc;
  }
  R[PHI] -= u * gpx + v * gpy;
  R[PSI] = -(u * gsx + v * gsy);
  R[RE] -= comp;
  if (prm.gravity) {
    R[RU] += rho * pf.gx;
    R[RV] += rho * pf.gy;
    R[RE] += rho * (pf.gx * u + pf.gy * v);
  }
  if (ST) {
    const float s = pf.sigma * kappa * sqrtf(gpx * gpx + gpy * gpy);
    R[RU] += s * nx;
    R[RV] += s * ny;
    R[RE] += s * (u * nx + v * ny);
  }
  if (act) store_node32<!VISC>(rvol, n, N, R);

  const bool onW = i == 0, onE = i == P;
  const bool onS = DIM == 2 && j == 0, onN = DIM == 2 && j == P;
  if (act && (onW || onE || onS || onN)) {
    const long base = (long)e * NFK;
    // the sound speed, with the reader's former operations (trace_derive)
    const float cs = VISC ? 0.f : sqrtf((Pr + (Pr + fmaf(pf.dC, phi, pf.C2)) * iG) * ir);
    auto put = [&](int f, int kk, float gn, float nn, float t1, float t2) {
      if (!in_bounds(prm.status, base + f * NK + kk, (long long)prm.E * NFK)) return;
      float4 *rec = reinterpret_cast<float4 *>(tr) + (base + f * NK + kk) * (TRW32 / 4);
      rec[0] = make_float4(q[0], q[1], q[2], q[3]);
      rec[1] = make_float4(q[4], q[5], q[6], gn);
      rec[2] = VISC ? make_float4(nn, t1, t2, 0.f) : make_float4(nn, Pr, cs, ir);
    };
    const int kx = DIM == 2 ? j : 0;
    if (onW) put(0, kx, gpx, nx, txx, txy);
    if (onE) put(1, kx, gpx, nx, txx, txy);
    if (onS) put(2, i, gpy, ny, txy, tyy);
    if (onN) put(3, i, gpy, ny, txy, tyy);
  }
}

// PDL (here and in the kernels below): launched as a programmatic dependent of
// the kernel before (launch_dependent).
template <int P, int DIM, bool VISC, bool ST, bool PDL>
__global__ void __launch_bounds__(Geom<P, DIM, VISC, ST>::THREADS)
k_volume32(const Params prm, const ParamsF pf, const float *__restrict__ opsf, const float *__restrict__ w,
           float *__restrict__ rvol, float *__restrict__ tr, const double *__restrict__ w64,
           float *__restrict__ w32out, float *__restrict__ lo_out, double *__restrict__ w64copy) {
  constexpr int P11 = Geom<P, DIM, VISC, ST>::P1 * Geom<P, DIM, VISC, ST>::P1;
  __shared__ float s_op[2 * P11];  // Dx, Dy
  if (PDL) {
    grid_dependents_launch();
    for (int t = threadIdx.x; t < 2 * P11; t += blockDim.x) s_op[t] = opsf[t];
    grid_dependency_wait();
  }
  vol32_body<P, DIM, VISC, ST, 0, PDL>(prm, pf, opsf, s_op, PDL, blockIdx.x, w, rvol, tr, w64, w32out, nullptr,
                                       lo_out, w64copy);
}

// The NC words of face-trace record o (records of RW floats, 128-bit loads), or, when the record
// does not exist, zeros with m1 = m1_default (a finite density for the closure).
template <int NC, int RW, bool COH = false>
__device__ __forceinline__ void load_trace32(const float *__restrict__ tr, long o, bool valid, float *T,
                                             float m1_default) {
#pragma unroll
  for (int qf = 0; qf < NC; ++qf) T[qf] = qf == T_M1 ? m1_default : 0.f;
  if (!valid) return;
  const float4 *rec = reinterpret_cast<const float4 *>(tr) + o * (RW / 4);
#pragma unroll
  for (int k = 0; k < (NC + 3) / 4; ++k) {
    const float4 x = ld_in<COH>(rec + k);
    if (4 * k + 0 < NC) T[4 * k + 0] = x.x;
    if (4 * k + 1 < NC) T[4 * k + 1] = x.y;
    if (4 * k + 2 < NC) T[4 * k + 2] = x.z;
    if (4 * k + 3 < NC) T[4 * k + 3] = x.w;
  }
}

// Surface kernel body of the FP32-bulk path.  mode MODE_RHS writes L for the
// paper's variables in FP64 (io.out64, with L(rho E) = L(rhoEt) + (C_1-C_2) L(phi));
// the stage modes write the stage increment (MODE_S1, MODE_S2: io.dout) or add
// the last increment to the step start in float-float (MODE_S3) and write the
// new step start (io.hi_out, io.lo_out), or, when io.out64 is given, the FP64
// state (last stage of a call).  See StageIO.
//
// s_op: the block's shared copy of the operator table (OpsLayout, Geom::OPS
// floats), filled by this body.
//
// rout != NULL (stage modes): the stage state of the thread's node (step start
// plus increment, in FP32; for MODE_S3 the new step start's hi part) is also
// left in rout, for a volume body that follows in the same kernel.  Every
// thread of the block returns from this body (none leaves early), so such a
// body may synchronise the block.
// PDL: the kernel was launched as a programmatic dependent; the operator table
// is copied before the wait for the kernel before, whose results are then read
// with coherent loads.
// FUSED: the body runs in a fused stage kernel (modes MODE_S1..MODE_S3 with hi_out / lo_out), so the
// FP64 outputs (MODE_RHS, out64, w64in) are compiled out of it.
// FMAP: how face nodes are given to threads (below): 1 block-level, 0 element-level, -1 the default
// (block-level in 2D at p = 1, 4, 5).
template <int P, int DIM, bool VISC, bool ST, int EPBX = 0, bool PDL = false, bool FUSED = false, int FMAP = -1>
__device__ __forceinline__ void surf32_body(const Params &prm, const ParamsF &pf, const float *__restrict__ opsf,
                                            float *s_op, int blk, int mode, float dt, const StageIO &io,
                                            const float *__restrict__ rvol, const float *__restrict__ tr,
                                            float *rout = nullptr) {
  using G = Geom<P, DIM, VISC, ST, EPBX>;
  constexpr int P1 = G::P1, NP = G::NP, EPB = G::EPB, NFK = G::NFK, NK = G::NK;
  constexpr int RW = TRW32;                          // floats per trace record
  constexpr int NC = VISC ? NT32_VISCOUS : TRW32;    // words read per trace record
  // Face nodes to threads.  Block-level: the block's EPB * NFK face nodes go to consecutive threads
  // (face node g = tid + fi * THREADS: element g / NFK, its face node g % NFK), so that the face
  // phase occupies as few warps as it can -- at p = 5 (120 face nodes, 192 threads) four warps
  // instead of all six, at p = 2 (84 face nodes, 64 threads) one warp for the second pass instead
  // of both: the batched ensemble's step 7.86 -> 7.61 ms, 64 x 64 p1 16.5 -> 15.7 us, the p = 4
  // surface kernels 4% faster, outputs bit-identical.  Element-level: the threads of an element
  // take its own face nodes (face node a + fi * NP), which stays faster for the 1D slab (8.7 vs
  // 9.8 us a step: its face nodes then spread over both warps of a block) and for single problems
  // at p = 2 (128 x 128: 12.4 vs 14.4 us per fused launch).  At p = 3 (NFK = NP, EPB * NP threads)
  // the two give the same assignment.
  constexpr bool BMAP = FMAP >= 0 ? FMAP == 1 : (DIM == 2 && P != 2 && P != 3);
  constexpr int NFC = EPB * NFK;
  constexpr int FPT = BMAP ? (NFC + G::THREADS - 1) / G::THREADS : (NFK + NP - 1) / NP;  // per thread
  const OpsLayout L{P1, NP};
  // Per face node: the surface integrand of the 7 equations (padded to 8 floats)
  // and the 6 lifting coefficients, in planes of consecutive face nodes, so that
  // the face nodes' 128- and 64-bit accesses are consecutive in shared memory.
  __shared__ float4 s_surf[2][EPB][NFK];
  __shared__ float4 s_lift0[EPB][NFK];
  __shared__ float2 s_lift1[EPB][NFK];

  const int le_raw = threadIdx.x / NP;
  const bool lane = le_raw < EPB;
  const int le = lane ? le_raw : EPB - 1;
  const int a = threadIdx.x % NP;
  const int e = blk * EPB + le;
  const int N = prm.N;
  const bool act = lane && e < prm.E && in_bounds(prm.status, (long long)e * NP + a, N);
  const long n = (long)(act ? e : 0) * NP + a;

  int e2_[FPT];  // neighbour across the face of each face node (-1: wall)
  // block-level: face node fi of the thread -- its element's slot fle in the block, index t within the
  // element (NFK: none), element fe; true when the face node exists
  auto face_of = [&](int fi, int &fle, int &t, int &fe) {
    const int g = threadIdx.x + fi * G::THREADS;
    fle = g < NFC ? g / NFK : 0;
    t = g < NFC ? g % NFK : NFK;
    fe = blk * EPB + fle;
    return g < NFC && fe < prm.E;
  };
  if (PDL) {
#pragma unroll
    for (int fi = 0; fi < FPT; ++fi) {
      if constexpr (BMAP) {
        int fle, t, fe;
        const bool fv = face_of(fi, fle, t, fe);
        e2_[fi] = fv ? neighbour(prm, fe, t / NK) : -1;
      } else {
        const int t = a + fi * NP;
        e2_[fi] = act && t < NFK ? neighbour(prm, e, t / NK) : -1;
      }
    }
    for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = opsf[t];
    grid_dependency_wait();
  }

  // Every global load of the body is issued first -- the node's own inputs of
  // the update and both traces of its face nodes -- so that their latencies
  // overlap each other (and the copy of the operator table).
  float Lv[NV], w0n[NV], dn[NV], lon[NV];
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) Lv[vv] = w0n[vv] = dn[vv] = lon[vv] = 0.f;
  double w64n[NV];
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) w64n[vv] = 0.0;
  const bool fp64_start = !FUSED && mode == MODE_S3 && io.w64in != nullptr;
  if (act) {
    load_node32<!VISC, PDL>(rvol, n, N, Lv);
    if (mode != MODE_RHS && !fp64_start) load_node32<!VISC, PDL>(io.w0, n, N, w0n);
    if (mode == MODE_S2 || mode == MODE_S3) load_node32<!VISC, PDL>(io.din, n, N, dn);
    if (mode == MODE_S3 && !fp64_start) load_node32<!VISC, PDL>(io.lo, n, N, lon);
    if (fp64_start) {
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) w64n[vv] = ld_in<PDL>(io.w64in + (long)vv * N + n);
    }
  }
  float Cm_[FPT][NC], Cp_[FPT][NC];
#pragma unroll
  for (int fi = 0; fi < FPT; ++fi) {
    int t, fe;
    bool fv;
    if constexpr (BMAP) {
      int fle;
      fv = face_of(fi, fle, t, fe);
    } else {
      t = a + fi * NP;
      fv = act && t < NFK;
      fe = e;
    }
    const int f = fv ? t / NK : 0, kk = fv ? t % NK : 0;
    const int e2 = PDL ? e2_[fi] : (fv ? neighbour(prm, fe, f) : -1);
    e2_[fi] = e2;
    const long om = (long)(BMAP ? (fv ? fe : 0) : (act ? e : 0)) * NFK + (fv ? t : 0);
    const long op = (long)(e2 >= 0 ? e2 : 0) * NFK + (f ^ 1) * NK + kk;
    const long long ntr = (long long)prm.E * NFK;
    load_trace32<NC, RW, PDL>(tr, om, fv && in_bounds(prm.status, om, ntr), Cm_[fi], 1.f);
    load_trace32<NC, RW, PDL>(tr, op, e2 >= 0 && in_bounds(prm.status, op, ntr), Cp_[fi], 0.f);
  }

  if (!PDL)
    for (int t = threadIdx.x; t < L.size(); t += blockDim.x) s_op[t] = opsf[t];
  __syncthreads();
  const float *Dx = s_op + L.Dx(), *Dy = s_op + L.Dy();
  const float *invM = s_op + L.invM(), *wfx = s_op + L.wfx(), *wfy = s_op + L.wfy();
  if (io.dt_dev) dt = (float)ld_in<PDL>(io.dt_dev);

#pragma unroll
  for (int fi = 0; fi < FPT; ++fi) {
    int fle, t;
    if constexpr (BMAP) {
      int fe;
      face_of(fi, fle, t, fe);
      if (t >= NFK) continue;
    } else {
      t = a + fi * NP;
      if (!lane || t >= NFK) continue;
      fle = le;
    }
    const int f = t / NK, kk = t % NK;
    const bool wall = e2_[fi] < 0;
    const bool xf = f < 2;
    const float sg = (f & 1) ? 1.f : -1.f;
    float Tm[NT_VISCOUS], Tp[NT_VISCOUS];
#pragma unroll
    for (int qf = 0; qf < NV; ++qf) Tm[qf] = Cm_[fi][qf];
    Tm[T_GPHI] = Cm_[fi][C_GPHI];
    Tm[T_N] = Cm_[fi][C_N];
    if (VISC) {
      Tm[T_TX] = Cm_[fi][C_TX];
      Tm[T_TY] = Cm_[fi][C_TY];
    }
    if (VISC) trace_derive<DIM, VISC>(pf, Tm);
    else trace_stored<DIM>(pf, Cm_[fi], Tm);
    if (!wall) {
#pragma unroll
      for (int qf = 0; qf < NV; ++qf) Tp[qf] = Cp_[fi][qf];
      Tp[T_GPHI] = Cp_[fi][C_GPHI];
      Tp[T_N] = Cp_[fi][C_N];
      if (VISC) {
        Tp[T_TX] = Cp_[fi][C_TX];
        Tp[T_TY] = Cp_[fi][C_TY];
        trace_derive<DIM, VISC>(pf, Tp);
      } else {
        trace_stored<DIM>(pf, Cp_[fi], Tp);
      }
    } else {
#pragma unroll
      for (int qf = 0; qf < NT_VISCOUS; ++qf) Tp[qf] = Tm[qf];
      if (prm.bc[f] == BC_SLIP) {
        if (xf) { Tp[T_RU] = -Tm[T_RU]; Tp[T_U] = -Tm[T_U]; }
        else    { Tp[T_RV] = -Tm[T_RV]; Tp[T_V] = -Tm[T_V]; }
      } else if (prm.bc[f] == BC_PRESSURE) {
        // exterior state at rest at p_bc: the reduced energy is p_bc times the mixture 1/(gamma-1)
        Tp[T_RU] = Tp[T_RV] = 0.f;
        Tp[T_RE] = (float)prm.p_bc[f] * fmaf(Tp[T_PHI], pf.g1 - pf.g2, pf.g2);
        trace_derive<DIM, VISC>(pf, Tp);
      } else {
        Tp[T_RU] = -Tm[T_RU]; Tp[T_U] = -Tm[T_U];
        Tp[T_RV] = -Tm[T_RV]; Tp[T_V] = -Tm[T_V];
      }
    }
    const float mx = xf ? sg : 0.f, my = xf ? 0.f : sg;
    const float unm = Tm[T_U] * mx + Tm[T_V] * my;
    const float unp = Tp[T_U] * mx + Tp[T_V] * my;
    const float lam = fmaxf(fabsf(unm) + Tm[T_C], fabsf(unp) + Tp[T_C]);
    const float wf = xf ? wfx[kk] : wfy[kk];

    float S[NV];
    {
      const float Fm[5] = {Tm[T_M1] * unm, Tm[T_M2] * unm, Tm[T_RU] * unm + Tm[T_P] * mx,
                           Tm[T_RV] * unm + Tm[T_P] * my, (Tm[T_RE] + Tm[T_P]) * unm};
      const float Fp[5] = {Tp[T_M1] * unp, Tp[T_M2] * unp, Tp[T_RU] * unp + Tp[T_P] * mx,
                           Tp[T_RV] * unp + Tp[T_P] * my, (Tp[T_RE] + Tp[T_P]) * unp};
#pragma unroll
      for (int c = 0; c < 5; ++c) {  // F- - F^ = (F- - F+)/2 + lambda [[w]]
        const int vv = M1 + c;
        S[vv] = wf * (0.5f * (Fm[c] - Fp[c]) + lam * 0.5f * (Tp[vv] - Tm[vv]));
      }
    }
    // compression term on the face: -1/2 Cmix(phi+) (u+ - u-) . m
    S[RE] -= wf * 0.5f * fmaf(pf.dC, Tp[T_PHI], pf.C2) * (unp - unm);
    S[PHI] = wf * (lam - unm) * 0.5f * (Tp[T_PHI] - Tm[T_PHI]);
    S[PSI] = wf * (lam - unm) * 0.5f * (Tp[T_PSI] - Tm[T_PSI]);

    float lift[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    {
      // SIP flux minus the own trace of the a_1 flux, for every a_1-derived term:
      // C^ a^.m - C- a-.m (at a wall no a_1 flux crosses: a^ = 0)
      const float km = 0.5f * (Tm[T_U] * Tm[T_U] + Tm[T_V] * Tm[T_V]);
      const float a1m = pf.Gamma * (pf.eps * Tm[T_GPHI] - Tm[T_PHI] * (1.f - Tm[T_PHI]) * Tm[T_N]) * sg;
      const float Co[6] = {1.f, pf.rho01, -pf.rho02, pf.drho0 * Tm[T_U], pf.drho0 * Tm[T_V],
                           Tm[T_B] + pf.drho0 * km};
      const int slot[6] = {PHI, M1, M2, RU, RV, RE};
      if (!wall) {
        const float eta = xf ? pf.eta_x : pf.eta_y;
        const float jump = Tp[T_PHI] - Tm[T_PHI];
        const float gn = 0.5f * (Tp[T_GPHI] + Tm[T_GPHI]) * sg;
        const float sharp =
            0.5f * (Tp[T_PHI] * (1.f - Tp[T_PHI]) * Tp[T_N] + Tm[T_PHI] * (1.f - Tm[T_PHI]) * Tm[T_N]) * sg;
        const float ahat = pf.Gamma * (pf.eps * (gn + eta * jump) - sharp);
        const float kp = 0.5f * (Tp[T_U] * Tp[T_U] + Tp[T_V] * Tp[T_V]);
        const float Cq[6] = {1.f, pf.rho01, -pf.rho02, pf.drho0 * 0.5f * (Tp[T_U] + Tm[T_U]),
                             pf.drho0 * 0.5f * (Tp[T_V] + Tm[T_V]),
                             0.5f * (Tp[T_B] + Tm[T_B]) + pf.drho0 * 0.5f * (kp + km)};
        const float sym = -wf * 0.5f * pf.Gamma * pf.eps * jump;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          S[slot[c]] += wf * (Cq[c] * ahat - Co[c] * a1m);
          lift[c] = Cq[c] * sym;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) S[slot[c]] -= wf * Co[c] * a1m;
      }
    }
    if (VISC) {
      const float eta = xf ? pf.eta_x : pf.eta_y;
      const float mua = 0.5f * (Tp[T_MU] + Tm[T_MU]);
      const float tmx = Tm[T_TX] * sg, tmy = Tm[T_TY] * sg;
      const float tpx = Tp[T_TX] * sg, tpy = Tp[T_TY] * sg;
      // tau^ . m - tau- . m
      S[RU] += wf * (0.5f * (tpx - tmx) + eta * mua * (Tp[T_U] - Tm[T_U]));
      S[RV] += wf * (0.5f * (tpy - tmy) + eta * mua * (Tp[T_V] - Tm[T_V]));
      const float km = 0.5f * (Tm[T_U] * Tm[T_U] + Tm[T_V] * Tm[T_V]);
      const float kp = 0.5f * (Tp[T_U] * Tp[T_U] + Tp[T_V] * Tp[T_V]);
      const float tum = tmx * Tm[T_U] + tmy * Tm[T_V];
      const float tup = tpx * Tp[T_U] + tpy * Tp[T_V];
      S[RE] += wf * (0.5f * (tup - tum) + eta * mua * (kp - km));
    }
    s_surf[0][fle][t] = make_float4(S[0], S[1], S[2], S[3]);
    s_surf[1][fle][t] = make_float4(S[4], S[5], S[6], 0.f);
    s_lift0[fle][t] = make_float4(lift[0], lift[1], lift[2], lift[3]);
    s_lift1[fle][t] = make_float2(lift[4], lift[5]);
  }
  __syncthreads();

  if (act) {
    const int i = a % P1, j = DIM == 2 ? a / P1 : 0;
    float acc[NV] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto face_add = [&](int f, int kk) {
      const float4 x = s_surf[0][le][f * NK + kk], y = s_surf[1][le][f * NK + kk];
      acc[0] += x.x; acc[1] += x.y; acc[2] += x.z; acc[3] += x.w;
      acc[4] += y.x; acc[5] += y.y; acc[6] += y.z;
    };
    const int kx = DIM == 2 ? j : 0;
    if (i == 0) face_add(0, kx);
    if (i == P) face_add(1, kx);
    if (DIM == 2 && j == 0) face_add(2, i);
    if (DIM == 2 && j == P) face_add(3, i);
    {
      // the symmetric SIP term of the four faces, weighted by the boundary row of D
      auto lift_add = [&](int fn, float wgt) {
        const float4 x = s_lift0[le][fn];
        const float2 y = s_lift1[le][fn];
        acc[PHI] += x.x * wgt;
        acc[M1] += x.y * wgt;
        acc[M2] += x.z * wgt;
        acc[RU] += x.w * wgt;
        acc[RV] += y.x * wgt;
        acc[RE] += y.y * wgt;
      };
      lift_add(0 * NK + kx, -Dx[0 * P1 + i]);
      lift_add(1 * NK + kx, Dx[P * P1 + i]);
      if (DIM == 2) {
        lift_add(2 * NK + i, -Dy[0 * P1 + j]);
        lift_add(3 * NK + i, Dy[P * P1 + j]);
      }
    }
    const float im = invM[a];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) Lv[vv] += acc[vv] * im;
    bool bad = false;
    if (!FUSED && mode == MODE_RHS) {
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) {
        double r = f2d(Lv[vv]);
        if (vv == RE) r = fma(prm.dC, f2d(Lv[PHI]), r);
        bad |= !isfinite(r);
        io.out64[(long)vv * N + n] = r;
      }
    } else {
      float r[NV];
      if (fp64_start) {
        // w_{n+1} = w_n + 2 (d2 + dt L) / 3 in FP64 on the caller's state; the increment of the
        // reduced energy becomes one of rho E by adding (C_1 - C_2) times that of phi
        float d[NV];
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) {
          d[vv] = (2.f / 3.f) * fmaf(dt, Lv[vv], dn[vv]);
          bad |= !isfinite(d[vv]);
          r[vv] = 0.f;
        }
#pragma unroll
        for (int vv = 0; vv < RE; ++vv) io.out64[(long)vv * N + n] = w64n[vv] + f2d(d[vv]);
        io.out64[(long)RE * N + n] = w64n[RE] + fma(prm.dC, f2d(d[PHI]), f2d(d[RE]));
      } else if (mode == MODE_S3) {
        // w_{n+1} = (hi, lo) + 2 (d2 + dt L) / 3, in float-float
        float lo[NV];
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) {
          r[vv] = w0n[vv];
          lo[vv] = lon[vv];
          ff_add(r[vv], lo[vv], (2.f / 3.f) * fmaf(dt, Lv[vv], dn[vv]));
          bad |= !isfinite(r[vv]);
        }
        if (!FUSED && io.out64) {
          // last stage of a call: hand back the FP64 state hi + lo, restoring the stiffened-gas
          // constant with the carried phi
#pragma unroll
          for (int vv = 0; vv < RE; ++vv) io.out64[(long)vv * N + n] = ff_to_double(r[vv], lo[vv]);
          const double phi64 = ff_to_double(r[PHI], lo[PHI]);
          io.out64[(long)RE * N + n] = ff_to_double(r[RE], lo[RE]) + fma(prm.dC, phi64, prm.C2);
        } else {
          store_node32<!VISC>(io.hi_out, n, N, r);
          store_node32<!VISC>(io.lo_out, n, N, lo);
        }
      } else {
        // d1 = dt L,  d2 = (d1 + dt L) / 4; the stage state is w0 + d
        float d[NV];
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) {
          d[vv] = mode == MODE_S1 ? dt * Lv[vv] : 0.25f * fmaf(dt, Lv[vv], dn[vv]);
          r[vv] = w0n[vv] + d[vv];
          bad |= !isfinite(r[vv]);
        }
        store_node32<!VISC>(io.dout, n, N, d);
      }
      if (rout) {
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) rout[vv] = r[vv];
      }
    }
    if (prm.check_finite && bad) atomicOr(prm.status, STATUS_NONFINITE);
  }
}

template <int P, int DIM, bool VISC, bool ST, bool PDL>
__global__ void __launch_bounds__(Geom<P, DIM, VISC, ST>::THREADS)
k_surface32(const Params prm, const ParamsF pf, const float *__restrict__ opsf, int mode, float dt, const StageIO io,
            const float *__restrict__ rvol, const float *__restrict__ tr) {
  __shared__ float s_op[Geom<P, DIM, VISC, ST>::OPS];
  if (PDL) grid_dependents_launch();
  surf32_body<P, DIM, VISC, ST, 0, PDL>(prm, pf, opsf, s_op, blockIdx.x, mode, dt, io, rvol, tr);
}

// Fused stage kernel: the surface part of stage s (mode MODE_S1..S3) followed,
// in the same block, by the volume part of stage s+1 on the stage result.
// The surface part of an element needs the face traces of its neighbours, so
// it cannot follow the volume part of the same stage inside one launch; the
// volume part of the next stage needs only the element's own new state, which
// the thread of each node already holds.  So a step of SSP-RK3 is one volume
// launch and three fused launches (and three fused launches per step when
// several steps run back to back), and the stage state is handed from one
// part to the other in registers.  The volume part and the traces go to the
// other buffer of a pair (rvol_out, tr_out), because neighbouring blocks of
// the same launch may still read rvol_in and tr_in.
// Residency of the viscous variants and of every variant at p >= 4: at most 72 registers a thread
// (65,536 / (THREADS x 72) CTAs per SM: 7 of 128 threads at p = 4).  Uncapped, the viscous
// surface-tension variant needs 90 and runs 6% slower at p = 4 than at 80; at 72 it spills a few
// words and runs 2% faster than at 80, and at 64 (more spills) no faster than at 80.  The inviscid
// p = 4 variants fit 72 without spills and run 18% faster than uncapped (86 vs 105 us at 256 x 256).
// Below p = 4 the inviscid grids of the single-problem workloads are one partial wave, where
// residency does not bind.
template <int P, int DIM, bool VISC, bool ST, bool PDL>
__global__ void __launch_bounds__(Geom<P, DIM, VISC, ST>::THREADS,
                                  (VISC || P >= 4) ? 65536 / (Geom<P, DIM, VISC, ST>::THREADS * 72) : 1)
k_surfvol32(const Params prm, const ParamsF pf, const float *__restrict__ opsf, int mode, float dt, const StageIO io,
            const float *__restrict__ rvol_in, const float *__restrict__ tr_in, float *__restrict__ rvol_out,
            float *__restrict__ tr_out) {
  __shared__ float s_op[Geom<P, DIM, VISC, ST>::OPS];  // one table for both parts
  float r[NV];
  if (PDL) grid_dependents_launch();
  surf32_body<P, DIM, VISC, ST, 0, PDL, true>(prm, pf, opsf, s_op, blockIdx.x, mode, dt, io, rvol_in, tr_in, r);
  vol32_body<P, DIM, VISC, ST>(prm, pf, opsf, s_op, true, blockIdx.x, nullptr, rvol_out, tr_out, nullptr, nullptr,
                               r);
}

// Launch interface of one FP32-bulk kernel family.  volume: the volume part of a
// stage on the FP32 state w, or, with w64, on the FP64 state, which it splits
// into the internal state's hi (w32out) and lo (lo_out, may be NULL) parts and
// copies into w64copy (may be NULL).
struct KernelSet32 {
  cudaError_t (*volume)(const Params &, const ParamsF &, const float *opsf, const float *w, float *rvol,
                        float *trace, const double *w64, float *w32out, float *lo_out, double *w64copy,
                        cudaStream_t);
  cudaError_t (*surface)(const Params &, const ParamsF &, const float *opsf, int mode, float dt, const StageIO &io,
                         const float *rvol, const float *trace, cudaStream_t);
  cudaError_t (*surfvol)(const Params &, const ParamsF &, const float *opsf, int mode, float dt, const StageIO &io,
                         const float *rvol_in, const float *tr_in, float *rvol_out, float *tr_out, cudaStream_t);
  int nt, epb, threads;
};

// A grid that the device holds at once is launched as a programmatic dependent
// of the kernel before it: its launch, CTA start and operator-table copy
// overlap that kernel's tail, which is most of the gain on latency-bound
// stages (64x64 p3: 4.9 instead of 6.2 us per volume launch back to back).  A
// grid of several waves gains nothing from an early start, and the early CTAs
// of the next kernel would take the places where this grid's later waves
// balance over the SMs, so it is launched plainly (and reads with the
// non-coherent loads, a few per cent faster on the viscous surface kernels).
template <int P, int DIM, bool VISC, bool ST>
cudaError_t launch_volume32(const Params &prm, const ParamsF &pf, const float *opsf, const float *w, float *rvol,
                            float *trace, const double *w64, float *w32out, float *lo_out, double *w64copy,
                            cudaStream_t s) {
  using G = Geom<P, DIM, VISC, ST>;
  const int blocks = (prm.E + G::EPB - 1) / G::EPB;
  static const int resident = resident_blocks(k_volume32<P, DIM, VISC, ST, true>, G::THREADS);
  if (blocks <= resident)
    return launch_dependent(k_volume32<P, DIM, VISC, ST, true>, blocks, G::THREADS, s, prm, pf, opsf, w, rvol,
                            trace, w64, w32out, lo_out, w64copy);
  k_volume32<P, DIM, VISC, ST, false><<<blocks, G::THREADS, 0, s>>>(prm, pf, opsf, w, rvol, trace, w64, w32out,
                                                                    lo_out, w64copy);
  return cudaGetLastError();
}

template <int P, int DIM, bool VISC, bool ST>
cudaError_t launch_surface32(const Params &prm, const ParamsF &pf, const float *opsf, int mode, float dt,
                             const StageIO &io, const float *rvol, const float *trace, cudaStream_t s) {
  using G = Geom<P, DIM, VISC, ST>;
  const int blocks = (prm.E + G::EPB - 1) / G::EPB;
  static const int resident = resident_blocks(k_surface32<P, DIM, VISC, ST, true>, G::THREADS);
  if (blocks <= resident)
    return launch_dependent(k_surface32<P, DIM, VISC, ST, true>, blocks, G::THREADS, s, prm, pf, opsf, mode,
                            dt, io, rvol, trace);
  k_surface32<P, DIM, VISC, ST, false><<<blocks, G::THREADS, 0, s>>>(prm, pf, opsf, mode, dt, io, rvol, trace);
  return cudaGetLastError();
}

template <int P, int DIM, bool VISC, bool ST>
cudaError_t launch_surfvol32(const Params &prm, const ParamsF &pf, const float *opsf, int mode, float dt,
                             const StageIO &io, const float *rvol_in, const float *tr_in, float *rvol_out,
                             float *tr_out, cudaStream_t s) {
  using G = Geom<P, DIM, VISC, ST>;
  const int blocks = (prm.E + G::EPB - 1) / G::EPB;
  static const int resident = resident_blocks(k_surfvol32<P, DIM, VISC, ST, true>, G::THREADS);
  if (blocks <= resident)
    return launch_dependent(k_surfvol32<P, DIM, VISC, ST, true>, blocks, G::THREADS, s, prm, pf, opsf, mode,
                            dt, io, rvol_in, tr_in, rvol_out, tr_out);
  k_surfvol32<P, DIM, VISC, ST, false><<<blocks, G::THREADS, 0, s>>>(prm, pf, opsf, mode, dt, io, rvol_in, tr_in,
                                                                     rvol_out, tr_out);
  return cudaGetLastError();
}

template <int P, int DIM, bool VISC, bool ST>
KernelSet32 make_set32() {
  using G = Geom<P, DIM, VISC, ST>;
  return KernelSet32{&launch_volume32<P, DIM, VISC, ST>, &launch_surface32<P, DIM, VISC, ST>,
                     &launch_surfvol32<P, DIM, VISC, ST>, VISC ? NT32_VISCOUS : NT32_INVISCID, G::EPB,
                     G::THREADS};
}

template <int P>
bool kernels_fp32_p(int dim, bool viscous, bool st, KernelSet32 *out) {
  if (dim == 1) {
    if (viscous || st) return false;
    *out = make_set32<P, 1, false, false>();
    return true;
  }
  if (!viscous && !st) *out = make_set32<P, 2, false, false>();
  else if (viscous && !st) *out = make_set32<P, 2, true, false>();
  else if (!viscous && st) *out = make_set32<P, 2, false, true>();
  else *out = make_set32<P, 2, true, true>();
  return true;
}

bool kernels_fp32(int p, int dim, bool viscous, bool surface_tension, KernelSet32 *out);

}  // namespace dgpf
