// Explicit instantiation of the FP64 kernel families of order p = 1.
#include "dg_kernels_fp64.cuh"

namespace dgpf {
bool kernels_fp64_p1(int dim, bool viscous, bool st, KernelSet *out) {
  return kernels_fp64_p<1>(dim, viscous, st, out);
}
}  // namespace dgpf
