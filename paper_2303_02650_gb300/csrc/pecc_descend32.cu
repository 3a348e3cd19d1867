// pecc_descend32.cu -- the binary32 instances of the descent kernel (own translation unit, so that
// they compile in parallel with the others).
#include "pecc_descend_kernel.cuh"

namespace pecc {

// 512 threads with 128 registers; 128-thread blocks with 96 registers (five per SM, no spills) and
// with 80 registers (six per SM, a few spilled bytes).
static const DescendVariant kVar32[] = {descend_variant<Arith32, 512, 1>(), descend_variant<Arith32, 128, 5>(),
                                        descend_variant<Arith32, 128, 6>()};

int descend_variants32(const DescendVariant **v) {
  *v = kVar32;
  return (int)(sizeof(kVar32) / sizeof(kVar32[0]));
}

}  // namespace pecc
