// Explicit instantiation of the adjoint kernels of order p = 2.
#include "dg_adjoint.cuh"

namespace dgpf {
bool adj_kernels_p2(int dim, AdjKernels *out) { return adj_kernels_p<2>(dim, out); }
}  // namespace dgpf
