// Explicit instantiation of the FP64 kernel families of order p = 4.
#include "dg_kernels_fp64.cuh"

namespace dgpf {
bool kernels_fp64_p4(int dim, bool viscous, bool st, KernelSet *out) {
  return kernels_fp64_p<4>(dim, viscous, st, out);
}
}  // namespace dgpf
