// Explicit instantiation of the adjoint kernels of order p = 3.
#include "dg_adjoint.cuh"

namespace dgpf {
bool adj_kernels_p3(int dim, AdjKernels *out) { return adj_kernels_p<3>(dim, out); }
}  // namespace dgpf
