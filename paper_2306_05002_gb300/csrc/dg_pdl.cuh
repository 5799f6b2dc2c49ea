// dg_pdl.cuh -- programmatic dependent launch for the FP32-bulk stage kernels
// of libdgpf (GB300, sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace dgpf {

// Programmatic dependent launch (sm_90 and later).  A kernel started with
// launch_dependent() may be scheduled while the kernel before it on the stream
// is still running, so that its launch, its CTAs' start and its prologue (index
// arithmetic, the operator tables, which nothing writes after creation) overlap
// that kernel's tail.  Before its first access to memory that an earlier
// kernel reads or writes, every thread calls grid_dependency_wait(), which
// returns once the earlier kernel has completed and its writes are visible.
// grid_dependents_launch() lets the next kernel be scheduled early.  Both are
// no-ops in a kernel launched without the attribute.  Data that an earlier
// kernel writes is read with coherent loads (ld.global.ca, __ldca), never with
// the non-coherent ld.global.nc (__ldg): that form declares the data read-only
// for the whole life of the kernel, which stops being true once the kernel
// overlaps its predecessor, and nothing then orders it after the wait.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Blocks of `kernel` (at `threads` a block) that the device holds at once.
template <typename K>
inline int resident_blocks(K kernel, int threads) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess)
    return 0;
  return nsm * per;
}

// Launch with the programmatic-serialization attribute.
template <typename... K, typename... A>
inline cudaError_t launch_dependent(void (*kernel)(K...), int blocks, int threads, cudaStream_t s, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace dgpf
