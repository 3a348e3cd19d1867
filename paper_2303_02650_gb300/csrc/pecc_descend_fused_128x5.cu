// pecc_descend_fused_128x5.cu -- the fused descent kernel compiled for at most 128 threads per block and
// 5 resident blocks per SM (its register budget).
#include "pecc_descend_kernel.cuh"

namespace pecc {
DescendVariant descend_fused_128x5() { return descend_fused_variant<128, 5>(); }
}  // namespace pecc
