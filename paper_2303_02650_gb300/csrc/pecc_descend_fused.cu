// pecc_descend_fused.cu -- the fused instances of the descent kernel: the FP32 descent and the FP64
// polish of each instance back to back in one block.  Each instance is compiled in a translation
// unit of its own (pecc_descend_fused_*.cu), so that they compile in parallel.
#include "pecc_internal.h"

namespace pecc {

// 128 registers (two 256-thread or four 128-thread blocks per SM), 96 (five 128-thread blocks), and
// one 512-thread block per SM (a few large instances, each block alone on its SM).
static const DescendVariant kVarFused[] = {descend_fused_256x2(), descend_fused_128x5(), descend_fused_512x1()};

int descend_variants_fused(const DescendVariant **v) {
  *v = kVarFused;
  return (int)(sizeof(kVarFused) / sizeof(kVarFused[0]));
}

cudaError_t launch_descend_fused(const DescendVariant &v, const DescendParams &p32, const DescendParams &p64, int grid,
                                 int block, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (block > v.max_threads) return cudaErrorInvalidValue;
  void *args[] = {(void *)&p32, (void *)&p64};
  return cudaLaunchKernel(v.fn, dim3(grid), dim3(block), args, p32.smem_bytes, s);
}

}  // namespace pecc
