// Tile variants of the batched FP32-bulk kernels of order p = 2.
#include "dg_batch.cuh"

namespace dgpf {
void batch_variants_p2(BatchVariant *out) { batch_variants_p<2>(out); }
}  // namespace dgpf
