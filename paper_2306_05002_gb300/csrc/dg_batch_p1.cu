// Tile variants of the batched FP32-bulk kernels of order p = 1.
#include "dg_batch.cuh"

namespace dgpf {
void batch_variants_p1(BatchVariant *out) { batch_variants_p<1>(out); }
}  // namespace dgpf
