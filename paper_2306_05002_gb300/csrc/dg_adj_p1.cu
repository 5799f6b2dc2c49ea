// Explicit instantiation of the adjoint kernels of order p = 1.
#include "dg_adjoint.cuh"

namespace dgpf {
bool adj_kernels_p1(int dim, AdjKernels *out) { return adj_kernels_p<1>(dim, out); }
}  // namespace dgpf
