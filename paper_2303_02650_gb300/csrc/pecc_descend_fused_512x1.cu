// pecc_descend_fused_512x1.cu -- the fused descent kernel compiled for at most 512 threads per block and
// 1 resident block per SM (its register budget).
#include "pecc_descend_kernel.cuh"

namespace pecc {
DescendVariant descend_fused_512x1() { return descend_fused_variant<512, 1>(); }
}  // namespace pecc
