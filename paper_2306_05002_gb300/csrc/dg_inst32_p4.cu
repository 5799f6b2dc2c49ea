// Explicit instantiation of the FP32-bulk kernel families of order p = 4.
#include "dg_kernels_fp32.cuh"

namespace dgpf {
bool kernels_fp32_p4(int dim, bool viscous, bool st, KernelSet32 *out) {
  return kernels_fp32_p<4>(dim, viscous, st, out);
}
}  // namespace dgpf
