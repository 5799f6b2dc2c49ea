// Explicit instantiation of the FP64 kernel families of order p = 3.
#include "dg_kernels_fp64.cuh"

namespace dgpf {
bool kernels_fp64_p3(int dim, bool viscous, bool st, KernelSet *out) {
  return kernels_fp64_p<3>(dim, viscous, st, out);
}
}  // namespace dgpf
