// Explicit instantiation of the adjoint kernels of order p = 5.
#include "dg_adjoint.cuh"

namespace dgpf {
bool adj_kernels_p5(int dim, AdjKernels *out) { return adj_kernels_p<5>(dim, out); }
}  // namespace dgpf
