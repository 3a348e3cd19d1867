// pecc_descend_fused_256x2.cu -- the fused descent kernel compiled for at most 256 threads per block and
// 2 resident blocks per SM (its register budget).
#include "pecc_descend_kernel.cuh"

namespace pecc {
DescendVariant descend_fused_256x2() { return descend_fused_variant<256, 2>(); }
}  // namespace pecc
