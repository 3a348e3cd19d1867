// pecc_tc.cuh -- fifth-generation tensor core helpers (tcgen05, TMEM) for the learned part's MLP.
//
// Operands live in shared memory without swizzle, as "core matrices" of 8 rows x 16 bytes (8 bf16),
// each row's 16 bytes contiguous.  A matrix stored [r][c] (c fastest within a core) puts core
// (r / 8, c / 8) at (r / 8) * SR + (c / 8) * 128 bytes, SR = (C / 8) * 128.  One such buffer
// serves as a K-major operand (K = c) and as an MN-major operand (K = r): in the shared-memory
// descriptor the leading byte offset is always the stride between cores adjacent along K and the
// stride byte offset the stride between cores adjacent along M or N.  The accumulator of an
// M = 128 MMA holds row m in TMEM lane m and column n in TMEM column base + n (32-bit each); warp
// w of the block reads lanes 32 w .. 32 w + 31.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace pecc {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, c) in the core layout of a matrix with C columns (C a multiple of 8).
__host__ __device__ __forceinline__ uint32_t core_off(int r, int c, int C) {
  return (uint32_t)((r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Shared-memory descriptor: no swizzle, descriptor version 1 (bits 46-47), base offset 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Operand descriptors of the core layout of a matrix with C columns starting at addr:
// K along the columns (K-major) or K along the rows (MN-major).
__device__ __forceinline__ uint64_t desc_k_cols(uint32_t addr, int C) { return sdesc(addr, 128, (uint32_t)(C >> 3) * 128); }
__device__ __forceinline__ uint64_t desc_k_rows(uint32_t addr, int C) { return sdesc(addr, (uint32_t)(C >> 3) * 128, 128); }

// Instruction descriptor of kind::f16 with bf16 A and B, f32 accumulator; a_mn / b_mn: the operand
// is MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = (acc ? D : 0) + A B^T for one K = 16 step; issued by one thread.
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The mbarrier receives one arrival when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of phase `parity` of the mbarrier, for at most limit_ns; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long long limit_ns) {
  const long long t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
    if (now_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor cores' reads
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one whole warp; the address goes to *dst (shared memory).
template <int NCOL> __device__ __forceinline__ void tmem_alloc(uint32_t *dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "n"(NCOL));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
template <int NCOL> __device__ __forceinline__ void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOL));
}

// 32 consecutive 32-bit columns of this thread's lane (warp w reads lanes 32 w ..); the load and
// its wait are one asm statement, so no use of the registers can move above the wait.
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc
}  // namespace pecc
