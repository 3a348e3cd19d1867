// pecc_mlp.cu -- the learned warm start: a per-circle MLP that reads the relative offsets of a
// circle's 12 nearest neighbours and its distance to the container wall and proposes a
// displacement; training (forward, backward, Adam) and inference are the kernels below, with the
// 128-wide GEMMs of every layer on the fifth-generation tensor cores (tcgen05.mma, BF16 inputs,
// FP32 accumulators in TMEM).
//
// Features of circle i (binary32, every operation correctly rounded so that a plain CPU
// restatement reproduces them bit for bit): the frame e_r = c_i / |c_i| (e_r = (1, 0) at the
// origin), e_t = (-e_r.y, e_r.x); the 12 nearest other centres within 4.5 (by squared distance,
// then index) as offsets d = c_j - c_i projected on (e_r, e_t), zero where fewer exist; and
// b = min(R - |c_i| - 1, 4.5).  The network 25 -> 128 -> 128 -> 128 -> 2 (ReLU) outputs the
// displacement in the same frame.
#include <cuda_bf16.h>

#include "pecc_internal.h"
#include "pecc_tc.cuh"

namespace pecc {
namespace {

using bf16 = __nv_bfloat16;

constexpr int KNN = 12;
constexpr float kKnnR2 = 4.5f * 4.5f;
constexpr int H = 128;
constexpr int F = 25;      // features
constexpr int SA = 136;    // padded row stride (bf16) of 128-wide tiles: conflict-free fragments
constexpr int S1 = 40;     // padded row stride of 32-wide tiles

// ---------------------------------------------------------------------------- parameters ----
// Flat binary32 parameter vector: W1[128][25] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
// W4[2][128] b4[2].
constexpr int OW1 = 0, OB1 = OW1 + H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + 2 * H, NPAR = OB4 + 2;
// BF16 copies in the padded layouts the kernels read: W1[128][40] W2[128][136] W3[128][136] W4[16][136].
constexpr int BW1 = 0, BW2 = BW1 + H * S1, BW3 = BW2 + H * SA, BW4 = BW3 + H * SA, NBW = BW4 + 16 * SA;

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}


// ------------------------------------------------------------------------------- features ----
__device__ __forceinline__ float2 frame_er(float2 c) {
  const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(c.x, c.x), __fmul_rn(c.y, c.y)));
  if (!(r > 0.f)) return make_float2(1.f, 0.f);
  return make_float2(__fdiv_rn(c.x, r), __fdiv_rn(c.y, r));
}

// One block per instance: cell sort (grid side >= 2.5, so 4.5 is within two cells), then per
// circle the 12 nearest within 4.5 and the wall distance.
__global__ void features_kernel(StandaloneParams P, float *feat) {
  __shared__ int32_t sh[40];
  const int q = blockIdx.x;
  const InstDesc D = P.desc[q];
  const int n = D.n;
  const float2 *x = P.x32 + D.off;
  float2 *xs = (float2 *)P.xtmp + D.off;
  const CellGrid G{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
  uint32_t *ckey = P.ckey_t + D.off;
  int32_t *corder = P.corder_t + D.off;
  int32_t *cells = P.cells + D.cell_off;
  cta_cell_sort<float>(x, n, G, ckey, corder, cells, xs, sh);
  const int nc = G.nc;
  const float Rf = (float)D.R;
  for (int q0 = threadIdx.x; q0 < n; q0 += blockDim.x) {
    const int i = corder[q0];
    const float2 xi = xs[q0];
    const uint32_t key = ckey[i];
    const int cx = (int)(key % (uint32_t)nc), cy = (int)(key / (uint32_t)nc);
    float bs[KNN];
    int bj[KNN];
    float bx[KNN], by[KNN];
#pragma unroll
    for (int u = 0; u < KNN; ++u) { bs[u] = 3.0e38f; bj[u] = 0x7fffffff; bx[u] = 0.f; by[u] = 0.f; }
    const int bx0 = max(cx - 2, 0), bx1 = min(cx + 2, nc - 1);
    for (int yy = max(cy - 2, 0); yy <= min(cy + 2, nc - 1); ++yy) {
      const int lo = cells[yy * nc + bx0], hi = cells[yy * nc + bx1 + 1];
      for (int qq = lo; qq < hi; ++qq) {
        if (qq == q0) continue;
        const float2 xj = xs[qq];
        const float dx = __fsub_rn(xj.x, xi.x), dy = __fsub_rn(xj.y, xi.y);
        const float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (!(s < kKnnR2)) continue;
        const int j = corder[qq];
        if (s > bs[KNN - 1] || (s == bs[KNN - 1] && j > bj[KNN - 1])) continue;
        // insert (s, j) into the ascending list (compare-swap down the unrolled list)
        float cs = s, cxv = dx, cyv = dy;
        int cj = j;
#pragma unroll
        for (int u = 0; u < KNN; ++u) {
          const bool less = cs < bs[u] || (cs == bs[u] && cj < bj[u]);
          if (less) {
            float ts = bs[u], tx = bx[u], ty = by[u];
            int tj = bj[u];
            bs[u] = cs; bj[u] = cj; bx[u] = cxv; by[u] = cyv;
            cs = ts; cj = tj; cxv = tx; cyv = ty;
          }
        }
      }
    }
    const float2 er = frame_er(xi);
    float *f = feat + (size_t)(D.off + i) * F;
#pragma unroll
    for (int u = 0; u < KNN; ++u) {
      const bool has = bj[u] != 0x7fffffff;
      const float fu = has ? __fadd_rn(__fmul_rn(bx[u], er.x), __fmul_rn(by[u], er.y)) : 0.f;
      const float fv = has ? __fsub_rn(__fmul_rn(by[u], er.x), __fmul_rn(bx[u], er.y)) : 0.f;
      f[2 * u] = fu;
      f[2 * u + 1] = fv;
    }
    const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(xi.x, xi.x), __fmul_rn(xi.y, xi.y)));
    const float b = __fsub_rn(__fsub_rn(Rf, r), 1.0f);
    f[24] = fminf(b, 4.5f);
  }
}

// Target of circle i: its displacement from x_before to now, in the frame of x_before.
__global__ void targets_kernel(StandaloneParams P, const double *__restrict__ xbefore, float *target) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const float2 x0 = make_float2((float)xbefore[2 * gi], (float)xbefore[2 * gi + 1]);
  const float2 x1 = P.x32[gi];
  const float2 er = frame_er(x0);
  const float dx = __fsub_rn(x1.x, x0.x), dy = __fsub_rn(x1.y, x0.y);
  target[2 * gi] = __fadd_rn(__fmul_rn(dx, er.x), __fmul_rn(dy, er.y));
  target[2 * gi + 1] = __fsub_rn(__fmul_rn(dy, er.x), __fmul_rn(dx, er.y));
}

// ------------------------------------------------------------------ tensor-core network ----
// Both kernels below keep every weight and activation tile in shared memory in the core layout of
// pecc_tc.cuh and run the 128-wide GEMMs as tcgen05 MMAs (M = 128 rows of a tile, K = 16 per
// instruction) issued by thread 0, with FP32 accumulators in TMEM; thread t of the 128 owns row t
// of a tile (TMEM lane t) in every epilogue.  The 2-wide output layer and its gradient run on the
// CUDA cores inside the epilogues.
constexpr int TM = 128;                  // rows per tile
constexpr int FPAD = 32;                 // padded input width
constexpr uint32_t kW1B = TM * FPAD * 2;  // bytes of a [128][32] bf16 core tile
constexpr uint32_t kHB = TM * H * 2;      // bytes of a [128][128] bf16 core tile
constexpr long long kWaitNs = 2000000000ll;  // bound of every wait on the MMA barrier
constexpr uint32_t kColStep = 2 * 128;       // a K step of 16 along the columns: two cores

// weights of the block: W1 [128][32], W2, W3 [128][128] in the core layout, from the padded bf16
// copies; biases b1 b2 b3 [128], the output layer W4 [2][128] (bf16 values) and b4 [2] as floats
__device__ void tc_load_weights(const bf16 *__restrict__ wb, const float *__restrict__ params, unsigned char *w1,
                                unsigned char *w2, unsigned char *w3, float *fb) {
  for (int u = threadIdx.x; u < TM * (FPAD / 8); u += blockDim.x) {
    const int o = u / (FPAD / 8), c8 = u % (FPAD / 8);
    *(uint4 *)(w1 + tc::core_off(o, 8 * c8, FPAD)) = *(const uint4 *)(wb + BW1 + o * S1 + 8 * c8);
  }
  for (int u = threadIdx.x; u < TM * (H / 8); u += blockDim.x) {
    const int o = u / (H / 8), c8 = u % (H / 8);
    *(uint4 *)(w2 + tc::core_off(o, 8 * c8, H)) = *(const uint4 *)(wb + BW2 + o * SA + 8 * c8);
    *(uint4 *)(w3 + tc::core_off(o, 8 * c8, H)) = *(const uint4 *)(wb + BW3 + o * SA + 8 * c8);
  }
  for (int u = threadIdx.x; u < H; u += blockDim.x) {
    fb[u] = params[OB1 + u];
    fb[H + u] = params[OB2 + u];
    fb[2 * H + u] = params[OB3 + u];
    fb[3 * H + u] = __bfloat162float(wb[BW4 + u]);
    fb[4 * H + u] = __bfloat162float(wb[BW4 + SA + u]);
  }
  if (threadIdx.x < 2) fb[5 * H + threadIdx.x] = params[OB4 + threadIdx.x];
}

// row r of the tile's input: the 25 features of global row gr (zero past rows and past column 25)
__device__ __forceinline__ void tc_load_row(const float *__restrict__ feat, int64_t gr, int64_t rows, int r,
                                            unsigned char *x) {
#pragma unroll
  for (int c8 = 0; c8 < FPAD / 8; ++c8) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int c = 8 * c8 + 2 * h;
      const float a = (gr < rows && c < F) ? feat[gr * F + c] : 0.f;
      const float b = (gr < rows && c + 1 < F) ? feat[gr * F + c + 1] : 0.f;
      w[h] = pack2(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
    }
    *(uint4 *)(x + tc::core_off(r, 8 * c8, FPAD)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// 32 bf16 values of row r starting at column c0 of a [128][128] core tile
__device__ __forceinline__ void tc_store32(unsigned char *t, int r, int c0, const float (&v)[32]) {
#pragma unroll
  for (int c8 = 0; c8 < 4; ++c8) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)
      w[h] = pack2(__float2bfloat16_rn(v[8 * c8 + 2 * h]), __float2bfloat16_rn(v[8 * c8 + 2 * h + 1]));
    *(uint4 *)(t + tc::core_off(r, c0 + 8 * c8, H)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}
__device__ __forceinline__ float tc_get(const unsigned char *t, int r, int c, int C) {
  return __bfloat162float(*(const bf16 *)(t + tc::core_off(r, c, C)));
}

// Thread 0 issues D = A B^T over K (K / 16 MMAs) and commits them to the barrier.  The operand
// descriptors advance by `astep` / `bstep` bytes per K step of 16.
__device__ __forceinline__ void tc_gemm(uint32_t d, uint32_t a_addr, bool a_krows, int a_cols, uint32_t astep,
                                        uint32_t b_addr, bool b_krows, int b_cols, uint32_t bstep, int N, int K,
                                        bool accumulate) {
  const uint32_t id = tc::idesc_bf16(TM, N, a_krows ? 1 : 0, b_krows ? 1 : 0);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint32_t aa = a_addr + ks * astep, ba = b_addr + ks * bstep;
    const uint64_t ad = a_krows ? tc::desc_k_rows(aa, a_cols) : tc::desc_k_cols(aa, a_cols);
    const uint64_t bd = b_krows ? tc::desc_k_rows(ba, b_cols) : tc::desc_k_cols(ba, b_cols);
    tc::mma(d, ad, bd, id, (accumulate || ks > 0) ? 1 : 0);
  }
}

// Make this block's shared-memory writes visible to the tensor cores and order TMEM accesses around
// a block barrier.
__device__ __forceinline__ void tc_sync() {
  tc::fence_smem_to_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

// Thread 0 commits the MMAs issued so far and waits for them; every thread learns whether the wait
// ended in time (block-uniform).
__device__ __forceinline__ bool tc_commit_wait(uint64_t *mbar, uint32_t &phase, int *flag) {
  if (threadIdx.x == 0) {
    tc::commit(mbar);
    *flag = tc::mbar_wait(mbar, phase, kWaitNs) ? 0 : 1;
  }
  phase ^= 1u;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  return *flag == 0;
}

// Epilogue of a hidden layer: this thread's row of the accumulator plus bias, ReLU, rounded to bf16
// into tile `t` (and, if set, the rounded values to trace[0..128)); with w4, also the output layer
// o0 / o1 += h W4^T from the rounded values.
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t tacc, const float *bias, unsigned char *t, float *trace,
                                                   const float *w4, float &o0, float &o1) {
  const int r = threadIdx.x;
  for (int c0 = 0; c0 < H; c0 += 32) {
    float v[32];
    tc::ld32(tacc + ((uint32_t)(r & ~31) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __bfloat162float(__float2bfloat16_rn(fmaxf(v[j] + bias[c0 + j], 0.f)));
    if (t) tc_store32(t, r, c0, v);
    if (trace)
#pragma unroll
      for (int j = 0; j < 32; ++j) trace[c0 + j] = v[j];
    if (w4)
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        o0 = fmaf(v[j], w4[c0 + j], o0);
        o1 = fmaf(v[j], w4[H + c0 + j], o1);
      }
  }
}

constexpr uint32_t kFwdW1 = 0, kFwdW2 = kFwdW1 + kW1B, kFwdW3 = kFwdW2 + kHB, kFwdX = kFwdW3 + kHB,
                   kFwdH = kFwdX + kW1B, kFwdF = kFwdH + kHB, kFwdBar = kFwdF + (5 * H + 2) * 4 + 8;
constexpr size_t kFwdSmem = (size_t)kFwdBar + 16 + 1024;  // + the barrier, TMEM address, flag; + alignment slack

// Forward: out[rows][2] for rows of feat[rows][25]; trace (may be null): float[rows][3][128], the
// bf16 activations of the three hidden layers.  Persistent over tiles of 128 rows.
__global__ void __launch_bounds__(128, 1) forward_tc_kernel(const bf16 *__restrict__ wb, const float *__restrict__ params,
                                                             const float *__restrict__ feat, int64_t rows, float *out,
                                                             float *trace) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *w1 = sm + kFwdW1, *w2 = sm + kFwdW2, *w3 = sm + kFwdW3, *x = sm + kFwdX, *h = sm + kFwdH;
  float *fb = (float *)(sm + kFwdF);
  uint64_t *mbar = (uint64_t *)(sm + kFwdBar);
  uint32_t *tslot = (uint32_t *)(mbar + 1);
  int *flag = (int *)(tslot + 1);
  const int r = threadIdx.x;
  tc_load_weights(wb, params, w1, w2, w3, fb);
  if (r == 0) { tc::mbar_init(mbar); *flag = 0; }
  if (r < 32) tc::tmem_alloc<128>(tslot);
  tc_sync();
  const uint32_t tacc = *tslot;
  const uint32_t sw1 = tc::smem_u32(w1), sw2 = tc::smem_u32(w2), sw3 = tc::smem_u32(w3), sx = tc::smem_u32(x),
                 sh = tc::smem_u32(h);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t tiles = (rows + TM - 1) / TM;
  for (int64_t tl = blockIdx.x; tl < tiles && ok; tl += gridDim.x) {
    const int64_t gr = tl * TM + r;
    float *tr = (trace && gr < rows) ? trace + gr * 3 * H : nullptr;
    tc_load_row(feat, gr, rows, r, x);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sx, false, FPAD, kColStep, sw1, false, FPAD, kColStep, H, FPAD, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    float o0 = 0.f, o1 = 0.f;
    tc_hidden_epilogue(tacc, fb, h, tr, nullptr, o0, o1);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sh, false, H, kColStep, sw2, false, H, kColStep, H, H, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    tc_hidden_epilogue(tacc, fb + H, h, tr ? tr + H : nullptr, nullptr, o0, o1);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sh, false, H, kColStep, sw3, false, H, kColStep, H, H, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    tc_hidden_epilogue(tacc, fb + 2 * H, nullptr, tr ? tr + 2 * H : nullptr, fb + 3 * H, o0, o1);
    if (gr < rows) {
      out[gr * 2] = o0 + fb[5 * H];
      out[gr * 2 + 1] = o1 + fb[5 * H + 1];
    }
    tc::fence_before();
    __syncthreads();  // every row's TMEM reads precede the next tile's MMAs
    tc::fence_after();
  }
  if (!ok)  // the tensor cores did not answer in time: NaN outputs, nothing left waiting
    for (int64_t gr = (int64_t)blockIdx.x * TM + r; gr < rows; gr += (int64_t)gridDim.x * TM) {
      out[gr * 2] = out[gr * 2 + 1] = __int_as_float(0x7fc00000);
    }
  tc::fence_before();
  __syncthreads();
  if (r < 32) {
    tc::fence_after();
    tc::tmem_free<128>(tacc);
  }
}

// ------------------------------------------------------------------------------- training ----
// One block per SM, persistent over tiles of 128 rows: forward (keeping X, H1, H2, H3), then
//   dO = 2 (out - target) / rows (rounded to bf16);  dW4 += dO' H3, db4 += sum dO   (CUDA cores)
//   dZ3 = (dO W4) o [H3 > 0]                                                         (CUDA cores)
//   dW3 += dZ3' H2 (TMEM, across tiles);  dH2 = dZ3 W3;  dZ2 = dH2 o [H2 > 0]        (tensor cores)
//   dW2 += dZ2' H1;  dH1 = dZ2 W2;  dZ1 = dH1 o [H1 > 0];  dW1 += dZ1' X             (tensor cores)
//   db_l += column sums of dZ_l.  Every GEMM input is bf16 (dZ rounded like the activations).
// The gradient accumulators dW3, dW2, dW1 stay in TMEM until the block's last tile; the block then
// writes its partial gradient to part[block][NPAR] and its loss to loss_part[block].
// bwd_trace (may be null): float[rows][4][128], the bf16 dZ3, dZ2, dZ1 of every row, then its bf16
// dO (2 values) and its outputs (2 values).
constexpr uint32_t kTrW1 = 0, kTrW2 = kTrW1 + kW1B, kTrW3 = kTrW2 + kHB, kTrX = kTrW3 + kHB, kTrH1 = kTrX + kW1B,
                   kTrH2 = kTrH1 + kHB, kTrH3 = kTrH2 + kHB, kTrZ = kTrH3 + kHB, kTrF = kTrZ + kHB;
// floats after kTrF: biases and W4 (5 H + 2), dO [128][2], dW4 accumulator [2][128], bias gradient
// accumulators db1 db2 db3 [128] and db4 [2], the loss of each warp [4]
constexpr int kTrFdO = 5 * H + 2, kTrFdW4 = kTrFdO + 2 * TM, kTrFdb = kTrFdW4 + 2 * H, kTrFls = kTrFdb + 3 * H + 2,
              kTrFn = kTrFls + 4;
constexpr uint32_t kTrBar = kTrF + ((kTrFn * 4 + 15) & ~15);
constexpr size_t kTrainSmem = (size_t)kTrBar + 16 + 1024;

__global__ void __launch_bounds__(128, 1) train_tc_kernel(const bf16 *__restrict__ wb, const float *__restrict__ params,
                                                           const float *__restrict__ feat, const float *__restrict__ target,
                                                           int64_t rows, float *part, float *loss_part,
                                                           float *fwd_trace, float *bwd_trace) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *w1 = sm + kTrW1, *w2 = sm + kTrW2, *w3 = sm + kTrW3, *x = sm + kTrX;
  unsigned char *h1 = sm + kTrH1, *h2 = sm + kTrH2, *h3 = sm + kTrH3, *z = sm + kTrZ;
  float *fb = (float *)(sm + kTrF);
  float *dO = fb + kTrFdO, *adW4 = fb + kTrFdW4, *adb = fb + kTrFdb, *lsw = fb + kTrFls;
  uint64_t *mbar = (uint64_t *)(sm + kTrBar);
  uint32_t *tslot = (uint32_t *)(mbar + 1);
  int *flag = (int *)(tslot + 1);
  const int r = threadIdx.x, lane = r & 31, w = r >> 5;
  tc_load_weights(wb, params, w1, w2, w3, fb);
  for (int u = r; u < 2 * H + 3 * H + 2; u += blockDim.x) adW4[u] = 0.f;  // adW4 and adb are adjacent
  if (r == 0) { tc::mbar_init(mbar); *flag = 0; }
  if (r < 32) tc::tmem_alloc<512>(tslot);
  tc_sync();
  // TMEM columns: [0, 128) the layer accumulator, [128, 256) dW3, [256, 384) dW2, [384, 416) dW1
  const uint32_t tacc = *tslot, tdw3 = tacc + 128, tdw2 = tacc + 256, tdw1 = tacc + 384;
  const uint32_t lanes = (uint32_t)(r & ~31) << 16;
  const uint32_t sw1 = tc::smem_u32(w1), sw2 = tc::smem_u32(w2), sw3 = tc::smem_u32(w3), sx = tc::smem_u32(x);
  const uint32_t sh1 = tc::smem_u32(h1), sh2 = tc::smem_u32(h2), sz = tc::smem_u32(z);
  const uint32_t kRowStep = 2 * (H / 8) * 128;     // two 8-row core groups of a [128][128] tile
  const uint32_t kRowStepX = 2 * (FPAD / 8) * 128;  // of a [128][32] tile
  const float scale = 2.f / (float)rows;
  float lsum = 0.f;
  uint32_t phase = 0;
  bool ok = true, first = true;
  const int64_t tiles = (rows + TM - 1) / TM;
  for (int64_t tl = blockIdx.x; tl < tiles && ok; tl += gridDim.x) {
    const int64_t gr = tl * TM + r;
    float *ft = (fwd_trace && gr < rows) ? fwd_trace + gr * 3 * H : nullptr;
    float *bt = (bwd_trace && gr < rows) ? bwd_trace + gr * 4 * H : nullptr;
    // ---- forward
    tc_load_row(feat, gr, rows, r, x);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sx, false, FPAD, kColStep, sw1, false, FPAD, kColStep, H, FPAD, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    float o0 = 0.f, o1 = 0.f;
    tc_hidden_epilogue(tacc, fb, h1, ft, nullptr, o0, o1);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sh1, false, H, kColStep, sw2, false, H, kColStep, H, H, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    tc_hidden_epilogue(tacc, fb + H, h2, ft ? ft + H : nullptr, nullptr, o0, o1);
    tc_sync();
    if (r == 0) tc_gemm(tacc, sh2, false, H, kColStep, sw3, false, H, kColStep, H, H, false);
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    tc_hidden_epilogue(tacc, fb + 2 * H, h3, ft ? ft + 2 * H : nullptr, fb + 3 * H, o0, o1);
    // ---- output layer: dO of this row, rounded to bf16
    float d0 = 0.f, d1 = 0.f;
    if (gr < rows) {
      d0 = (o0 + fb[5 * H]) - target[gr * 2];
      d1 = (o1 + fb[5 * H + 1]) - target[gr * 2 + 1];
    }
    lsum += d0 * d0 + d1 * d1;
    const float g0 = __bfloat162float(__float2bfloat16_rn(d0 * scale));
    const float g1 = __bfloat162float(__float2bfloat16_rn(d1 * scale));
    dO[2 * r] = g0;
    dO[2 * r + 1] = g1;
    if (bt) {
      bt[3 * H] = g0;
      bt[3 * H + 1] = g1;
      bt[3 * H + 2] = o0 + fb[5 * H];
      bt[3 * H + 3] = o1 + fb[5 * H + 1];
    }
    // dZ3 of this row from dO and W4, masked by H3
    for (int c0 = 0; c0 < H; c0 += 32) {
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        const float dz = fmaf(g1, fb[4 * H + c], g0 * fb[3 * H + c]);
        v[j] = tc_get(h3, r, c, H) > 0.f ? __bfloat162float(__float2bfloat16_rn(dz)) : 0.f;
      }
      tc_store32(z, r, c0, v);
      if (bt)
#pragma unroll
        for (int j = 0; j < 32; ++j) bt[c0 + j] = v[j];
    }
    tc_sync();
    // dW3 += dZ3' H2 and dH2 = dZ3 W3 on the tensor cores; meanwhile dW4, db4 and db3 on the CUDA cores
    if (r == 0) {
      tc_gemm(tdw3, sz, true, H, kRowStep, sh2, true, H, kRowStep, H, TM, !first);
      tc_gemm(tacc, sz, false, H, kColStep, sw3, true, H, kRowStep, H, H, false);
    }
    {
      float s0 = 0.f, s1 = 0.f, sb3 = 0.f;
      for (int q = 0; q < TM; ++q) {
        const float hq = tc_get(h3, q, r, H);
        s0 = fmaf(dO[2 * q], hq, s0);
        s1 = fmaf(dO[2 * q + 1], hq, s1);
        sb3 += tc_get(z, q, r, H);
      }
      adW4[r] += s0;
      adW4[H + r] += s1;
      adb[2 * H + r] += sb3;
      if (r < 2) {
        float sb4 = 0.f;
        for (int q = 0; q < TM; ++q) sb4 += dO[2 * q + r];
        adb[3 * H + r] += sb4;
      }
    }
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    // dZ2 = dH2 o [H2 > 0]
    for (int c0 = 0; c0 < H; c0 += 32) {
      float v[32];
      tc::ld32(tacc + lanes + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        v[j] = tc_get(h2, r, c0 + j, H) > 0.f ? __bfloat162float(__float2bfloat16_rn(v[j])) : 0.f;
      tc_store32(z, r, c0, v);
      if (bt)
#pragma unroll
        for (int j = 0; j < 32; ++j) bt[H + c0 + j] = v[j];
    }
    tc_sync();
    if (r == 0) {
      tc_gemm(tdw2, sz, true, H, kRowStep, sh1, true, H, kRowStep, H, TM, !first);
      tc_gemm(tacc, sz, false, H, kColStep, sw2, true, H, kRowStep, H, H, false);
    }
    {
      float sb2 = 0.f;
      for (int q = 0; q < TM; ++q) sb2 += tc_get(z, q, r, H);
      adb[H + r] += sb2;
    }
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    // dZ1 = dH1 o [H1 > 0]
    for (int c0 = 0; c0 < H; c0 += 32) {
      float v[32];
      tc::ld32(tacc + lanes + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        v[j] = tc_get(h1, r, c0 + j, H) > 0.f ? __bfloat162float(__float2bfloat16_rn(v[j])) : 0.f;
      tc_store32(z, r, c0, v);
      if (bt)
#pragma unroll
        for (int j = 0; j < 32; ++j) bt[2 * H + c0 + j] = v[j];
    }
    tc_sync();
    if (r == 0) tc_gemm(tdw1, sz, true, H, kRowStep, sx, true, FPAD, kRowStepX, FPAD, TM, !first);
    {
      float sb1 = 0.f;
      for (int q = 0; q < TM; ++q) sb1 += tc_get(z, q, r, H);
      adb[r] += sb1;
    }
    if (!(ok = tc_commit_wait(mbar, phase, flag))) break;
    first = false;
  }
  // ---- the block's partial gradient
  float *gp = part + (size_t)blockIdx.x * NPAR;
  const float nanv = __int_as_float(0x7fc00000);
  if (ok && !first) {
    for (int c0 = 0; c0 < H; c0 += 32) {
      float v[32];
      tc::ld32(tdw3 + lanes + (uint32_t)c0, v);
      for (int j = 0; j < 32; ++j) gp[OW3 + r * H + c0 + j] = v[j];
      tc::ld32(tdw2 + lanes + (uint32_t)c0, v);
      for (int j = 0; j < 32; ++j) gp[OW2 + r * H + c0 + j] = v[j];
    }
    float v[32];
    tc::ld32(tdw1 + lanes, v);
    for (int j = 0; j < F; ++j) gp[OW1 + r * F + j] = v[j];
  } else {
    const float fill = ok ? 0.f : nanv;  // a block without tiles adds nothing
    for (int u = r; u < H * H; u += blockDim.x) { gp[OW3 + u] = fill; gp[OW2 + u] = fill; }
    for (int u = r; u < H * F; u += blockDim.x) gp[OW1 + u] = fill;
  }
  __syncthreads();
  for (int u = r; u < H; u += blockDim.x) {
    gp[OB1 + u] = ok ? adb[u] : nanv;
    gp[OB2 + u] = ok ? adb[H + u] : nanv;
    gp[OB3 + u] = ok ? adb[2 * H + u] : nanv;
    gp[OW4 + u] = ok ? adW4[u] : nanv;
    gp[OW4 + H + u] = ok ? adW4[H + u] : nanv;
  }
  if (r < 2) gp[OB4 + r] = ok ? adb[3 * H + r] : nanv;
  lsum = warp_sum(lsum);
  if (lane == 0) lsw[w] = lsum;
  tc::fence_before();
  __syncthreads();
  if (r == 0) loss_part[blockIdx.x] = ok ? lsw[0] + lsw[1] + lsw[2] + lsw[3] : nanv;
  if (r < 32) {
    tc::fence_after();
    tc::tmem_free<512>(tacc);
  }
}

// grad[p] = sum over blocks of part[b][p]; loss = sum of the blocks' losses / rows
__global__ void grad_reduce_kernel(const float *__restrict__ part, int nb, float *grad, const float *__restrict__ lp,
                                   int64_t rows, float *loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPAR) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * NPAR + p];
    grad[p] = s;
  }
  if (p == 0 && loss) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += lp[b];
    *loss = s / (float)rows;
  }
}

// bf16 padded index of parameter p (-1 for biases)
__device__ __forceinline__ int bf_index(int p) {
  if (p < OB1) return BW1 + (p / F) * S1 + (p % F);
  if (p >= OW2 && p < OB2) return BW2 + ((p - OW2) / H) * SA + (p - OW2) % H;
  if (p >= OW3 && p < OB3) return BW3 + ((p - OW3) / H) * SA + (p - OW3) % H;
  if (p >= OW4 && p < OB4) return BW4 + ((p - OW4) / H) * SA + (p - OW4) % H;
  return -1;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mhat / (sqrt(vhat) + eps)
__global__ void adam_kernel(float *params, float *m, float *v, const float *__restrict__ grad, bf16 *wb, float lr,
                            float b1c, float b2c) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPAR) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  const float w = params[p] - lr * (mm / b1c) / (sqrtf(vv / b2c) + 1e-8f);
  params[p] = w;
  const int bi = bf_index(p);
  if (bi >= 0) wb[bi] = __float2bfloat16_rn(w);
}

__global__ void sync_bf16_kernel(const float *__restrict__ params, bf16 *wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPAR) return;
  const int bi = bf_index(p);
  if (bi >= 0) wb[bi] = __float2bfloat16_rn(params[p]);
}

// He-uniform initial weights from Philox4x32-10 (key = seed, counter = (p, 0, 0, 1)), zero biases
__global__ void init_params_kernel(float *params, uint64_t seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPAR) return;
  int fan = 0;
  if (p < OB1) fan = F;
  else if ((p >= OW2 && p < OB2) || (p >= OW3 && p < OB3) || (p >= OW4 && p < OB4)) fan = H;
  float w = 0.f;
  if (fan > 0) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)p, 0u, 0u, 1u), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float u = (float)(r.x >> 8) * (1.0f / 16777216.0f);
    const float a = sqrtf(6.0f / (float)fan);
    w = (2.f * u - 1.f) * a;
    if (p >= OW4 && p < OB4) w *= 0.1f;  // small output layer: the first proposals stay small
  }
  params[p] = w;
}

// ------------------------------------------------------------------------------ warm start ----
// x += clip(du e_r + dv e_t, max_move) per circle; the old coordinates go to backup
__global__ void apply_kernel(StandaloneParams P, const float *__restrict__ dout, float2 *backup, float max_move) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const float2 x = P.x32[gi];
  backup[gi] = x;
  const float2 er = frame_er(x);
  const float du = dout[2 * gi], dv = dout[2 * gi + 1];
  float dx = du * er.x - dv * er.y, dy = du * er.y + dv * er.x;
  const float nrm = sqrtf(dx * dx + dy * dy);
  if (nrm > max_move) { dx *= max_move / nrm; dy *= max_move / nrm; }
  if (!isfinite(dx) || !isfinite(dy)) { dx = 0.f; dy = 0.f; }
  const float2 nx = make_float2(x.x + dx, x.y + dy);
  P.x32[gi] = nx;
  P.x64[gi] = make_double2((double)nx.x, (double)nx.y);
}

// keep the move of an instance only if its energy did not rise; accepted[q] counts kept rounds
__global__ void revert_kernel(StandaloneParams P, const float2 *__restrict__ backup, const double *__restrict__ Eb,
                              const double *__restrict__ Ea, int32_t *accepted) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const int q = P.inst_of[gi];
  const bool keep = Ea[q] <= Eb[q];
  if (!keep) {
    const float2 x = backup[gi];
    P.x32[gi] = x;
    P.x64[gi] = make_double2((double)x.x, (double)x.y);
  }
  if (accepted && gi == P.desc[q].off) accepted[q] += keep ? 1 : 0;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int mlp_num_params() { return NPAR; }
int mlp_num_bf16() { return NBW; }

cudaError_t mlp_init(float *params, bf16 *wb, uint64_t seed, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(wb, 0, sizeof(bf16) * NBW, s);
  if (e) return e;
  init_params_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(params, seed);
  sync_bf16_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(params, wb);
  return cudaGetLastError();
}

cudaError_t mlp_sync_bf16(const float *params, bf16 *wb, cudaStream_t s) {
  sync_bf16_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(params, wb);
  return cudaGetLastError();
}

cudaError_t mlp_features(const StandaloneParams &p, float *feat, cudaStream_t s) {
  if (p.num > 0) features_kernel<<<p.num, 256, 0, s>>>(p, feat);
  return cudaGetLastError();
}

cudaError_t mlp_targets(const StandaloneParams &p, const double *xbefore, float *target, cudaStream_t s) {
  if (p.total > 0) targets_kernel<<<nblk(p.total, 256), 256, 0, s>>>(p, xbefore, target);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const bf16 *wb, const float *params, const float *feat, int64_t rows, float *out, int sms,
                        cudaStream_t s, float *trace) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e) return e;
    attr = true;
  }
  if (rows <= 0) return cudaSuccess;
  const int64_t tiles = (rows + TM - 1) / TM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms);
  forward_tc_kernel<<<grid, TM, kFwdSmem, s>>>(wb, params, feat, rows, out, trace);
  return cudaGetLastError();
}

int mlp_train_blocks(int sms) { return sms; }

cudaError_t mlp_grad(const bf16 *wb, const float *params, const float *feat, const float *target, int64_t rows,
                     float *part, float *lpart, float *grad, float *loss, int sms, cudaStream_t s, float *fwd_trace,
                     float *bwd_trace) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e) return e;
    attr = true;
  }
  const int nb = mlp_train_blocks(sms);
  train_tc_kernel<<<nb, TM, kTrainSmem, s>>>(wb, params, feat, target, rows, part, lpart, fwd_trace, bwd_trace);
  grad_reduce_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(part, nb, grad, lpart, rows, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, float *m, float *v, const float *grad, bf16 *wb, float lr, int step,
                     cudaStream_t s) {
  const float b1c = 1.f - powf(0.9f, (float)step), b2c = 1.f - powf(0.999f, (float)step);
  adam_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(params, m, v, grad, wb, lr, b1c, b2c);
  return cudaGetLastError();
}

cudaError_t mlp_apply(const StandaloneParams &p, const float *dout, float2 *backup, float max_move, cudaStream_t s) {
  if (p.total > 0) apply_kernel<<<nblk(p.total, 256), 256, 0, s>>>(p, dout, backup, max_move);
  return cudaGetLastError();
}

cudaError_t mlp_revert(const StandaloneParams &p, const float2 *backup, const double *Eb, const double *Ea,
                       int32_t *accepted, cudaStream_t s) {
  if (p.total > 0) revert_kernel<<<nblk(p.total, 256), 256, 0, s>>>(p, backup, Eb, Ea, accepted);
  return cudaGetLastError();
}

}  // namespace pecc
