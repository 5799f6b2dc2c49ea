// dg_batch.cuh -- descriptor and launch interface of the batched FP32-bulk kernels.
#pragma once

#include "dg_kernels_fp32.cuh"

namespace dgpf {

// Everything one problem of a batch needs, read by the batched kernels from
// device memory (one entry per problem, grouped by order).
struct BatchProb {
  Params prm;
  ParamsF pf;
  const float *opsf;                        // FP32 operator table (OpsLayout)
  float *ws, *w1, *w2;                      // internal FP32 state and the two inner stages
  float *rvol[2], *tr[2];                   // volume part and face traces, double-buffered (fused stages)
  double *w64;                              // the caller's FP64 state (read at stage 1, written at stage 3)
  float dt;                                 // this problem's step size
  int block0;                               // first block of this problem in its order's grid
};

// Kernel kinds of a batched step: the volume part of stage 1, the fused
// surface part of stage s with the volume part of stage s+1 (s = 1, 2), and
// the surface part of stage 3.
enum BatchKind { BK_VOLUME = 0, BK_SURFVOL = 1, BK_SURFACE = 2 };

struct BatchKernels {
  cudaError_t (*launch)(int kind, const BatchProb *probs, const int *block0, int nprob, int stage, int nblocks,
                        cudaStream_t s);
  int epb;
};

bool batch_kernels(int p, BatchKernels *out);

}  // namespace dgpf
