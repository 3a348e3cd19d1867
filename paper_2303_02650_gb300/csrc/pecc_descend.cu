// pecc_descend.cu -- host side of the persistent descent kernel (pecc_descend_kernel.cuh): the
// compiled instances per arithmetic, launch, shared-memory sizing.  The binary64 and mixed
// (polish) instances are compiled here, the binary32 ones in pecc_descend32.cu.
#include "pecc_descend_kernel.cuh"

namespace pecc {

// Instances by arithmetic, the largest register budget first.  A block of the FP64 kernel needs
// about 225 registers per thread for its binary64 state (fewer spill); the polish and the FP32
// kernel run without spills at 96 registers, which lets five 128-thread blocks share an SM.
static const DescendVariant kVar64[] = {descend_variant<Arith64, 256, 1>()};
static const DescendVariant kVarMix[] = {descend_variant<ArithMix, 256, 2>(), descend_variant<ArithMix, 128, 5>()};

int descend_variants(int arith, const DescendVariant **v) {
  if (arith == 0) { *v = kVar64; return (int)(sizeof(kVar64) / sizeof(kVar64[0])); }
  if (arith == 1) return descend_variants32(v);
  if (arith == 3) return descend_variants_fused(v);
  *v = kVarMix;
  return (int)(sizeof(kVarMix) / sizeof(kVarMix[0]));
}

__global__ void stamp_kernel(long long *t0) { *t0 = globaltimer_ns(); }

cudaError_t launch_stamp(long long *t0, cudaStream_t s) {
  stamp_kernel<<<1, 1, 0, s>>>(t0);
  return cudaGetLastError();
}

cudaError_t launch_descend(const DescendVariant &v, const DescendParams &p, int grid, int block, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (block > v.max_threads) return cudaErrorInvalidValue;
  void *args[] = {(void *)&p};
  return cudaLaunchKernel(v.fn, dim3(grid), dim3(block), args, p.smem_bytes, s);
}

int descend_max_block(int arith) { return (arith == 1 || arith == 3) ? 512 : 256; }

// Shared-memory bytes without a global fallback: the per-warp partials of the first reduction of
// a batch step and the k batch rings.
size_t descend_smem_mandatory(int arith, int k, int block) {
  const size_t sc = arith == 0 ? 8 : 4;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  return al(sc * (size_t)(block / 32) * kPA) + al(4 * (size_t)k * kRingInts);
}

// Shared-memory bytes the working set of an instance of n circles (k batches, m secant pairs)
// asks for, in the order the kernel carves it.
size_t descend_smem_need(int arith, int n, int k, int ncx, int block, int m, bool outer) {
  const size_t pos = arith == 1 ? 8 : 16, vec = arith == 0 ? 16 : 8, sc = arith == 0 ? 8 : 4;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t cells = 4 * (2 * (size_t)ncx * ncx + 2);
  size_t b = descend_smem_mandatory(arith, k, block) + al(sc * (size_t)k * kBasis * kBasis) + al(pos * n) +
             al(4 * (size_t)(n + 1)) + (outer ? al(4 * (size_t)n) : 0) + al(2 * (size_t)(8 * n + 64)) +
             3 * al(vec * n) + 2 * al(pos * n) + (cells <= pos * (size_t)n ? 0 : al(cells)) +
             2 * al(vec * (size_t)(m + 1) * n) + (outer ? al(2 * (size_t)(kOuterPerCircle * n + 64)) : 0);
  return b;
}

}  // namespace pecc
