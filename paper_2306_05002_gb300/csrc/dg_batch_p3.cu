// Tile variants of the batched FP32-bulk kernels of order p = 3.
#include "dg_batch.cuh"

namespace dgpf {
void batch_variants_p3(BatchVariant *out) { batch_variants_p<3>(out); }
}  // namespace dgpf
