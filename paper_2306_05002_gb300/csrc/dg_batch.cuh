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
  float *ws, *w1, *w2, *rvol, *tr;          // internal FP32 state, stages, volume part, traces
  double *w64;                              // the caller's FP64 state (read at stage 1, written at stage 3)
  float dt;                                 // this problem's step size
  int block0;                               // first block of this problem in its order's grid
};

struct BatchKernels {
  cudaError_t (*launch)(bool volume, const BatchProb *probs, const int *block0, int nprob, int stage, int nblocks,
                        cudaStream_t s);
  int epb;
};

bool batch_kernels(int p, BatchKernels *out);

}  // namespace dgpf
