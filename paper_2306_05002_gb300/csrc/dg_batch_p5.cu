// Tile variants of the batched FP32-bulk kernels of order p = 5.
#include "dg_batch.cuh"

namespace dgpf {
void batch_variants_p5(BatchVariant *out) { batch_variants_p<5>(out); }
}  // namespace dgpf
