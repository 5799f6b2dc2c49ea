// dg_batch.cu -- batched FP32-bulk stage kernels: many independent DG problems
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
#include "dg_batch.cuh"

namespace dgpf {

__device__ __forceinline__ const BatchProb &stage_descriptor(const BatchProb *__restrict__ probs,
                                                             const int *__restrict__ block0, int nprob,
                                                             unsigned char *s_raw, int *s_k) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(block0 + mid) <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    *s_k = lo;
  }
  __syncthreads();
  const int *src = reinterpret_cast<const int *>(probs + *s_k);
  int *dst = reinterpret_cast<int *>(s_raw);
  for (int t = threadIdx.x; t < (int)(sizeof(BatchProb) / 4); t += blockDim.x) dst[t] = __ldg(src + t);
  __syncthreads();
  return *reinterpret_cast<const BatchProb *>(s_raw);
}

// Volume part of stage 1: reads the caller's FP64 state, writes the FP32
// state, the volume part and the traces (buffer 0).
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_volume32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, &s_k);
  const int blk = (int)blockIdx.x - b.block0;
  __shared__ float s_op[2 * (P + 1) * (P + 1)];
  vol32_body<P, 2, false, false>(b.prm, b.pf, b.opsf, s_op, false, blk, b.ws, b.rvol[0], b.tr[0], b.w64, b.ws);
}

// Surface part of stage `stage` (1 or 2) fused with the volume part of the
// next stage; stage s reads buffer s-1 of each pair and writes the other.
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_surfvol32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob, int stage) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, &s_k);
  const int blk = (int)blockIdx.x - b.block0;
  const int in = stage - 1, out = in ^ 1;
  __shared__ float s_op[Geom<P, 2, false, false>::OPS];
  float r[NV];
  surf32_body<P, 2, false, false>(b.prm, b.pf, b.opsf, s_op, blk, stage == 1 ? MODE_S1 : MODE_S2, b.dt, b.ws,
                                  stage == 1 ? b.ws : b.w1, b.rvol[in], b.tr[in], stage == 1 ? b.w1 : b.w2,
                                  nullptr, r);
  vol32_body<P, 2, false, false>(b.prm, b.pf, b.opsf, s_op, true, blk, nullptr, b.rvol[out], b.tr[out], nullptr,
                                 nullptr, r);
}

// Surface part of stage 3: writes the caller's FP64 state.
template <int P>
__global__ void __launch_bounds__(Geom<P, 2, false, false>::THREADS)
k_surface32_batch(const BatchProb *__restrict__ probs, const int *__restrict__ block0, int nprob) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(BatchProb)];
  __shared__ int s_k;
  const BatchProb &b = stage_descriptor(probs, block0, nprob, s_raw, &s_k);
  const int blk = (int)blockIdx.x - b.block0;
  __shared__ float s_op[Geom<P, 2, false, false>::OPS];
  surf32_body<P, 2, false, false>(b.prm, b.pf, b.opsf, s_op, blk, MODE_S3, b.dt, b.ws, b.w2, b.rvol[0], b.tr[0],
                                  nullptr, b.w64);
}

template <int P>
cudaError_t launch_batch(int kind, const BatchProb *probs, const int *block0, int nprob, int stage, int nblocks,
                         cudaStream_t s) {
  using G = Geom<P, 2, false, false>;
  if (kind == BK_VOLUME) k_volume32_batch<P><<<nblocks, G::THREADS, 0, s>>>(probs, block0, nprob);
  else if (kind == BK_SURFVOL) k_surfvol32_batch<P><<<nblocks, G::THREADS, 0, s>>>(probs, block0, nprob, stage);
  else k_surface32_batch<P><<<nblocks, G::THREADS, 0, s>>>(probs, block0, nprob);
  return cudaGetLastError();
}

bool batch_kernels(int p, BatchKernels *out) {
  switch (p) {
    case 1: *out = {&launch_batch<1>, Geom<1, 2, false, false>::EPB}; return true;
    case 2: *out = {&launch_batch<2>, Geom<2, 2, false, false>::EPB}; return true;
    case 3: *out = {&launch_batch<3>, Geom<3, 2, false, false>::EPB}; return true;
    case 4: *out = {&launch_batch<4>, Geom<4, 2, false, false>::EPB}; return true;
    case 5: *out = {&launch_batch<5>, Geom<5, 2, false, false>::EPB}; return true;
    default: return false;
  }
}

}  // namespace dgpf
