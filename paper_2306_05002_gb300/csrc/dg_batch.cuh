// dg_batch.cuh -- batched FP32-bulk stage kernels: many independent DG problems
// of one polynomial order advanced by a single launch per kernel.
//
// The grid is the concatenation of every problem's element tiles.  Block b
// finds its problem k by binary search over the per-problem first-block
// table, stages problem k's descriptor (closure constants, operator table,
// buffers, step size) in shared memory, and runs the same kernel body as the
// single-problem FP32-bulk path (dg_kernels_fp32.cuh) on its tile.  Problems
// of different size share a launch without padding; problems of different
// order go to different launches (one per order present).  A step is, per
// order, one volume launch, two fused launches (surface part of a stage and
// volume part of the next) and one surface launch.
//
// Tiles.  Each order is compiled in NVAR tile variants -- elements per block
// (the single-problem rule, or twice that) times register budget (the
// compiler's choice, or capped at 64 per thread through the minimum-blocks
// launch bound, which raises the resident warps) -- and the library times
// them on the actual batch before its first step (dg_batch_step).
#pragma once

#include "dg_kernels_fp32.cuh"

namespace dgpf {

// Everything one problem of a batch needs, read by the batched kernels from
// device memory (one entry per problem, grouped by order).
struct BatchProb {
  Params prm;
  ParamsF pf;
  const float *opsf;                        // FP32 operator table (OpsLayout)
  float *ws, *d1, *d2;                      // internal FP32 state (step start) and the two inner increments
  float *rvol[2], *tr[2];                   // volume part and face traces, double-buffered (fused stages)
  double *w64;                              // the caller's FP64 state (read at stage 1, written at stage 3)
  float dt;                                 // this problem's step size
};

// Kernel kinds of a batched step: the volume part of stage 1, the fused
// surface part of stage s with the volume part of stage s+1 (s = 1, 2), and
// the surface part of stage 3.
enum BatchKind { BK_VOLUME = 0, BK_SURFVOL = 1, BK_SURFACE = 2 };

constexpr int NVAR = 4;  // tile variants per order

struct BatchVariant {
  cudaError_t (*launch)(int kind, const BatchProb *probs, const int *block0, int nprob, int stage, int nblocks,
                        cudaStream_t s);
  int epb;      // elements per block
  int threads;  // threads per block
  int minb;     // minimum resident blocks per SM asked of the compiler (1: no register cap)
};

// The NVAR variants of order p (false if p is not available).
bool batch_variants(int p, BatchVariant *out);

// ---------------------------------------------------------------------------
// Kernel templates (instantiated per order in dg_batch_p<P>.cu).

// Find the block's problem (binary search over the first-block table) and
// stage its descriptor in shared memory; *blk receives the block's tile
// index within its problem.
__device__ __forceinline__ const BatchProb &stage_descriptor(const BatchProb *__restrict__ probs,
                                                             const int *__restrict__ block0, int nprob,
                                                             unsigned char *s_raw, int *s_k, int *blk) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(block0 + mid) <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_k[0] = lo;
    s_k[1] = (int)blockIdx.x - __ldg(block0 + lo);
  }
  __syncthreads();
  const int *src = reinterpret_cast<const int *>(probs + s_k[0]);
  int *dst = reinterpret_cast<int *>(s_raw);
  for (int t = threadIdx.x; t < (int)(sizeof(BatchProb) / 4); t += blockDim.x) dst[t] = __ldg(src + t);
  __syncthreads();
  *blk = s_k[1];
  return *reinterpret_cast<const BatchProb *>(s_raw);
}

template <int P, int EPBX>
using BGeom = Geom<P, 2, false, false, EPBX>;

// Volume part of stage 1: reads the caller's FP64 state, writes the FP32
// state, the volume part and the traces (buffer 0).
template <int P, int EPBX, int MINB>
__global__ void __launch_bounds__(BGeom<P, EPBX>::THREADS, MINB)
k_volume32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k[2];
  __shared__ float s_op[2 * (P + 1) * (P + 1)];
  int blk;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, s_k, &blk);
  vol32_body<P, 2, false, false, EPBX>(b.prm, b.pf, b.opsf, s_op, false, blk, b.ws, b.rvol[0], b.tr[0], b.w64,
                                       b.ws);
}

// Surface part of stage `stage` (1 or 2) fused with the volume part of the
// next stage; stage s reads buffer s-1 of each pair and writes the other.
// Stage 1 writes the increment d1, stage 2 reads it and writes d2.
template <int P, int EPBX, int MINB>
__global__ void __launch_bounds__(BGeom<P, EPBX>::THREADS, MINB)
k_surfvol32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob, int stage) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k[2];
  __shared__ float s_op[BGeom<P, EPBX>::OPS];
  int blk;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, s_k, &blk);
  const int in = stage - 1, out = in ^ 1;
  float r[NV];
  StageIO io{b.ws, nullptr, stage == 1 ? nullptr : b.d1, stage == 1 ? b.d1 : b.d2, nullptr, nullptr, nullptr,
             nullptr};
  surf32_body<P, 2, false, false, EPBX, false, true, 1>(b.prm, b.pf, b.opsf, s_op, blk, stage == 1 ? MODE_S1 : MODE_S2,
                                                     b.dt, io, b.rvol[in], b.tr[in], r);
  vol32_body<P, 2, false, false, EPBX>(b.prm, b.pf, b.opsf, s_op, true, blk, nullptr, b.rvol[out], b.tr[out],
                                       nullptr, nullptr, r);
}

// Surface part of stage 3: adds the last increment to the caller's FP64 state
// (the step start) in FP64, in place.
template <int P, int EPBX, int MINB>
__global__ void __launch_bounds__(BGeom<P, EPBX>::THREADS, MINB)
k_surface32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k[2];
  __shared__ float s_op[BGeom<P, EPBX>::OPS];
  int blk;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, s_k, &blk);
  StageIO io{nullptr, nullptr, b.d2, nullptr, nullptr, nullptr, b.w64, b.w64};
  surf32_body<P, 2, false, false, EPBX, false, false, 1>(b.prm, b.pf, b.opsf, s_op, blk, MODE_S3, b.dt, io, b.rvol[0],
                                                        b.tr[0]);
}

template <int P, int EPBX, int MINB>
cudaError_t launch_batch(int kind, const BatchProb *probs, const int *block0, int nprob, int stage, int nblocks,
                         cudaStream_t s) {
  constexpr int T = BGeom<P, EPBX>::THREADS;
  if (kind == BK_VOLUME) k_volume32_batch<P, EPBX, MINB><<<nblocks, T, 0, s>>>(probs, block0, nprob);
  else if (kind == BK_SURFVOL)
    k_surfvol32_batch<P, EPBX, MINB><<<nblocks, T, 0, s>>>(probs, block0, nprob, stage);
  else k_surface32_batch<P, EPBX, MINB><<<nblocks, T, 0, s>>>(probs, block0, nprob);
  return cudaGetLastError();
}

// Minimum blocks per SM that hold a block of T threads at 64 registers per thread.
constexpr int minb_cap64(int T) { return 65536 / (64 * T) > 1 ? 65536 / (64 * T) : 1; }

template <int P, int EPBX, int MINB>
BatchVariant make_variant() {
  return BatchVariant{&launch_batch<P, EPBX, MINB>, BGeom<P, EPBX>::EPB, BGeom<P, EPBX>::THREADS, MINB};
}

template <int P>
void batch_variants_p(BatchVariant *out) {
  constexpr int E1 = BGeom<P, 0>::EPB, E2 = 2 * E1;
  out[0] = make_variant<P, E1, 1>();
  out[1] = make_variant<P, E1, minb_cap64(BGeom<P, E1>::THREADS)>();
  out[2] = make_variant<P, E2, 1>();
  out[3] = make_variant<P, E2, minb_cap64(BGeom<P, E2>::THREADS)>();
}

}  // namespace dgpf
