// Explicit instantiation of the adjoint kernels of order p = 4.
#include "dg_adjoint.cuh"

namespace dgpf {
bool adj_kernels_p4(int dim, AdjKernels *out) { return adj_kernels_p<4>(dim, out); }
}  // namespace dgpf
