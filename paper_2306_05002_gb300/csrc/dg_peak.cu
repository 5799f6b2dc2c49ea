// dg_peak.cu -- dg_peak_flops: the FMA rate of the GPU's FP64 and FP32 pipes,
// measured by independent multiply-add chains, the denominators of the FP64
// path's rooflines (the FP32-bulk path is measured against the HBM copy rate).
#include <cuda_runtime.h>

#include "dgpf.h"

namespace {

constexpr int kChains = 8;    // independent chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

// Written only if the chains' sum took a value it cannot take (the chains
// converge to b / (1 - a)), so that the compiler keeps every multiply-add.
template <typename T>
__device__ T g_sink;

// Every thread advances kChains chains x <- x * a + b for `iters` rounds.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == (T)-1.2345e30) g_sink<T> = s;
}

template <typename T>
dg_status measure(int iters, double *tflops, cudaStream_t s) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_chains<T>, kThreads, 0);
  if (e != cudaSuccess || sms < 1 || per < 1) return DG_ERR_CUDA;
  const int blocks = sms * per;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return DG_ERR_CUDA;
  }
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters / 8 + 1, a, b);  // warm-up
  cudaEventRecord(ev[0], s);
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, a, b);
  cudaEventRecord(ev[1], s);
  e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return DG_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_peak_flops(int kind, int iters, double *tflops, void *stream) {
  if (!tflops || iters < 1 || (kind != 0 && kind != 1)) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return kind == 0 ? measure<double>(iters, tflops, s) : measure<float>(iters, tflops, s);
}
