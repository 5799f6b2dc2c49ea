// Tile variants of the batched FP32-bulk kernels of order p = 4.
#include "dg_batch.cuh"

namespace dgpf {
void batch_variants_p4(BatchVariant *out) { batch_variants_p<4>(out); }
}  // namespace dgpf
