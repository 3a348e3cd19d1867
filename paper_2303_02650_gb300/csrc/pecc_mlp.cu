// pecc_mlp.cu -- the learned warm start: a per-circle MLP that reads the relative offsets of a
// circle's 12 nearest neighbours and its distance to the container wall and proposes a
// displacement; training (forward, backward, Adam) and inference are the kernels below, with the
// three GEMMs of every layer on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulate).
//
// Features of circle i (binary32, every operation correctly rounded so that a plain CPU
// restatement reproduces them bit for bit): the frame e_r = c_i / |c_i| (e_r = (1, 0) at the
// origin), e_t = (-e_r.y, e_r.x); the 12 nearest other centres within 4.5 (by squared distance,
// then index) as offsets d = c_j - c_i projected on (e_r, e_t), zero where fewer exist; and
// b = min(R - |c_i| - 1, 4.5).  The network 25 -> 128 -> 128 -> 128 -> 2 (ReLU) outputs the
// displacement in the same frame.
#include <cuda_bf16.h>

#include "pecc_internal.h"

namespace pecc {
namespace {

using bf16 = __nv_bfloat16;

constexpr int KNN = 12;
constexpr float kKnnR2 = 4.5f * 4.5f;
constexpr int H = 128;
constexpr int F = 25;      // features
constexpr int FP = 32;     // padded input width
constexpr int SA = 136;    // padded row stride (bf16) of 128-wide tiles: conflict-free fragments
constexpr int S1 = 40;     // padded row stride of 32-wide tiles
constexpr int SO = 24;     // padded row stride of 16-wide tiles
constexpr int TR = 64;     // rows per block tile

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

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[16][8 NT] += A[16][K] B[K][8 NT] for one warp; A(m, k) = A[m * am + k * ak], B(k, n) = B[k * bk + n * bn]
// (shared memory, any strides: transposed operands are read in place).  Fragment layout of
// m16n8k16: lane = 4 g + t; A regs (g, 2t..), (g+8, 2t..), (g, 8+2t..), (g+8, 8+2t..); B regs
// (k = 2t.., n = g), (k = 8+2t.., n = g); C (g, 2t..), (g+8, 2t..).
template <int NT>
__device__ __forceinline__ void wgemm(float (&c)[NT][4], const bf16 *A, int am, int ak, const bf16 *B, int bk, int bn,
                                      int K) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * t, kb = ka + 8;
    const uint32_t a0 = pack2(A[g * am + ka * ak], A[g * am + (ka + 1) * ak]);
    const uint32_t a1 = pack2(A[(g + 8) * am + ka * ak], A[(g + 8) * am + (ka + 1) * ak]);
    const uint32_t a2 = pack2(A[g * am + kb * ak], A[g * am + (kb + 1) * ak]);
    const uint32_t a3 = pack2(A[(g + 8) * am + kb * ak], A[(g + 8) * am + (kb + 1) * ak]);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int nn = 8 * j + g;
      const uint32_t b0 = pack2(B[ka * bk + nn * bn], B[(ka + 1) * bk + nn * bn]);
      const uint32_t b1 = pack2(B[kb * bk + nn * bn], B[(kb + 1) * bk + nn * bn]);
      mma16816(c[j], a0, a1, a2, a3, b0, b1);
    }
  }
}

template <int NT> __device__ __forceinline__ void zero(float (&c)[NT][4]) {
#pragma unroll
  for (int j = 0; j < NT; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
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

// ------------------------------------------------------------------------- weights in smem ----
// biases in shared memory: b1[128] b2[128] b3[128] b4[2]
constexpr int SB1 = 0, SB2 = 128, SB3 = 256, SB4 = 384, NSB = 392;

__device__ void load_weights(const bf16 *__restrict__ wb, const float *__restrict__ params, bf16 *s, float *sb) {
  const uint4 *src = (const uint4 *)wb;
  uint4 *dst = (uint4 *)s;
  for (int u = threadIdx.x; u < NBW * 2 / 16; u += blockDim.x) dst[u] = src[u];
  for (int u = threadIdx.x; u < H; u += blockDim.x) {
    sb[SB1 + u] = params[OB1 + u];
    sb[SB2 + u] = params[OB2 + u];
    sb[SB3 + u] = params[OB3 + u];
  }
  if (threadIdx.x < 2) sb[SB4 + threadIdx.x] = params[OB4 + threadIdx.x];
}

// rows row0..row0+15 of the fp32 features [rows][25] into a bf16 [16][S1] tile (zero padded)
__device__ void load_x(const float *__restrict__ feat, int64_t row0, int64_t rows, bf16 *X) {
  for (int u = threadIdx.x & 31; u < 16 * FP; u += 32) {
    const int r = u / FP, c = u % FP;
    const int64_t gr = row0 + r;
    const float v = (gr < rows && c < F) ? feat[gr * F + c] : 0.f;
    X[r * S1 + c] = __float2bfloat16_rn(v);
  }
  __syncwarp();
}

// bias + ReLU on a warp's 16 x 128 accumulator, stored as bf16 into a [16][SA] tile
__device__ __forceinline__ void act_store(float (&c)[16][4], const float *__restrict__ bias, bf16 *Hs) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int col = 8 * j + 2 * t;
    const float b0 = bias[col], b1 = bias[col + 1];
    Hs[g * SA + col] = __float2bfloat16_rn(fmaxf(c[j][0] + b0, 0.f));
    Hs[g * SA + col + 1] = __float2bfloat16_rn(fmaxf(c[j][1] + b1, 0.f));
    Hs[(g + 8) * SA + col] = __float2bfloat16_rn(fmaxf(c[j][2] + b0, 0.f));
    Hs[(g + 8) * SA + col + 1] = __float2bfloat16_rn(fmaxf(c[j][3] + b1, 0.f));
  }
  __syncwarp();
}

// Forward of one warp's 16 rows; out[16][2] (fp32).  X, H1..H3: this warp's tiles.
__device__ void warp_forward(const bf16 *W, const float *sb, const bf16 *X, bf16 *H1, bf16 *H2, bf16 *H3,
                             float *out) {
  float c[16][4];
  zero(c);
  wgemm<16>(c, X, S1, 1, W + BW1, 1, S1, FP);
  act_store(c, sb + SB1, H1);
  zero(c);
  wgemm<16>(c, H1, SA, 1, W + BW2, 1, SA, H);
  act_store(c, sb + SB2, H2);
  zero(c);
  wgemm<16>(c, H2, SA, 1, W + BW3, 1, SA, H);
  act_store(c, sb + SB3, H3);
  float o[2][4];
  zero(o);
  wgemm<2>(o, H3, SA, 1, W + BW4, 1, SA, H);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (t == 0) {  // output columns 0 and 1 sit in n-tile 0 on the lanes with t == 0
    out[g * 2 + 0] = o[0][0] + sb[SB4];
    out[g * 2 + 1] = o[0][1] + sb[SB4 + 1];
    out[(g + 8) * 2 + 0] = o[0][2] + sb[SB4];
    out[(g + 8) * 2 + 1] = o[0][3] + sb[SB4 + 1];
  }
  __syncwarp();
}

constexpr size_t kWBytes = (size_t)NBW * 2;
constexpr size_t kHead = kWBytes + (size_t)NSB * 4;
constexpr size_t kFwdWarpBytes = (size_t)(16 * S1 + 3 * 16 * SA) * 2 + 16 * 2 * 4;
constexpr size_t kFwdSmem = kHead + 4 * kFwdWarpBytes;

__global__ void __launch_bounds__(128) forward_kernel(const bf16 *__restrict__ wb, const float *__restrict__ params,
                                                      const float *__restrict__ feat, int64_t rows, float *out) {
  extern __shared__ __align__(16) unsigned char sm[];
  bf16 *W = (bf16 *)sm;
  float *sb = (float *)(sm + kWBytes);
  load_weights(wb, params, W, sb);
  __syncthreads();
  const int w = threadIdx.x >> 5;
  unsigned char *mine = sm + kHead + (size_t)w * kFwdWarpBytes;
  bf16 *X = (bf16 *)mine, *H1 = X + 16 * S1, *H2 = H1 + 16 * SA, *H3 = H2 + 16 * SA;
  float *o = (float *)(H3 + 16 * SA);
  const int64_t tiles = (rows + 15) / 16;
  for (int64_t tl = (int64_t)blockIdx.x * 4 + w; tl < tiles; tl += (int64_t)gridDim.x * 4) {
    const int64_t r0 = tl * 16;
    load_x(feat, r0, rows, X);
    warp_forward(W, sb, X, H1, H2, H3, o);
    const int lane = threadIdx.x & 31;
    if (lane < 16 && r0 + lane < rows) {
      out[(r0 + lane) * 2] = o[lane * 2];
      out[(r0 + lane) * 2 + 1] = o[lane * 2 + 1];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------- training ----
// One block: 4 warps, tiles of 64 rows; forward (keeping X, H1..H3), then backward:
//   dO = 2 (out - target) / rows;  dW4 += dO' H3;  dZ3 = (dO W4) o [H3 > 0];  dW3 += dZ3' H2;
//   dZ2 = (dZ3 W3) o [H2 > 0];  dW2 += dZ2' H1;  dZ1 = (dZ2 W2) o [H1 > 0];  dW1 += dZ1' X;
//   db_l += column sums of dZ_l (db4 of dO).  GEMM inputs are bf16 (dZ rounded like the activations).
// Each block adds its tiles' gradients into its own binary32 slice part[block][NPAR].
constexpr size_t kTrainTile = (size_t)(TR * S1 + 3 * TR * SA + TR * SO + 2 * TR * SA) * 2 + TR * 2 * 4;
constexpr size_t kTrainSmem = kHead + kTrainTile;

// gp[base + (m0 + row) * ld + col] += accumulator of output rows m0.. (rows < mrows, cols < ncols)
template <int NT>
__device__ __forceinline__ void add_acc(float *gp, int base, int ld, const float (&c)[NT][4], int m0, int mrows,
                                        int ncols) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = 8 * j + 2 * t + h;
      if (col >= ncols) continue;
      if (m0 + g < mrows) gp[base + (m0 + g) * ld + col] += c[j][h];
      if (m0 + g + 8 < mrows) gp[base + (m0 + g + 8) * ld + col] += c[j][2 + h];
    }
  }
}

// dZ = (Zin Wl) o [Hmask > 0] for a warp's 16 rows (Zin: K columns), stored bf16 into Zout
__device__ __forceinline__ void back_layer(const bf16 *Zin, int zs, int K, const bf16 *Wl, const bf16 *Hmask, bf16 *Zout) {
  float c[16][4];
  zero(c);
  wgemm<16>(c, Zin, zs, 1, Wl, SA, 1, K);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int col = 8 * j + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool m0 = __bfloat162float(Hmask[g * SA + col + h]) > 0.f;
      const bool m1 = __bfloat162float(Hmask[(g + 8) * SA + col + h]) > 0.f;
      Zout[g * SA + col + h] = __float2bfloat16_rn(m0 ? c[j][h] : 0.f);
      Zout[(g + 8) * SA + col + h] = __float2bfloat16_rn(m1 ? c[j][2 + h] : 0.f);
    }
  }
  __syncwarp();
}

// dW[o][i] += sum_r Z[r][o] Hin[r][i] over the tile's 64 rows; warp w takes output rows 32w..32w+31
template <int NT>
__device__ __forceinline__ void weight_grad(float *gp, int base, int ld, const bf16 *Z, const bf16 *Hin, int hs,
                                            int ncols) {
  const int w = threadIdx.x >> 5;
  for (int mt = 2 * w; mt < 2 * w + 2; ++mt) {
    float c[NT][4];
    zero(c);
    wgemm<NT>(c, Z + 16 * mt, 1, SA, Hin, hs, 1, TR);
    add_acc<NT>(gp, base, ld, c, 16 * mt, H, ncols);
  }
}

__device__ __forceinline__ void bias_grad(float *gp, int base, const bf16 *Z) {
  for (int o = threadIdx.x; o < H; o += blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < TR; ++r) s += __bfloat162float(Z[r * SA + o]);
    gp[base + o] += s;
  }
}

__global__ void __launch_bounds__(128, 1) train_kernel(const bf16 *__restrict__ wb, const float *__restrict__ params,
                                                       const float *__restrict__ feat,
                                                       const float *__restrict__ target, int64_t rows, float *part,
                                                       float *loss_part) {
  extern __shared__ __align__(16) unsigned char sm[];
  bf16 *W = (bf16 *)sm;
  float *sb = (float *)(sm + kWBytes);
  unsigned char *tile = sm + kHead;
  bf16 *X = (bf16 *)tile;                  // [64][S1]
  bf16 *H1 = X + TR * S1;                  // [64][SA]
  bf16 *H2 = H1 + TR * SA;
  bf16 *H3 = H2 + TR * SA;
  bf16 *dO = H3 + TR * SA;                 // [64][SO]
  bf16 *Za = dO + TR * SO;                 // [64][SA]
  bf16 *Zb = Za + TR * SA;
  float *out = (float *)(Zb + TR * SA);    // [64][2]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  load_weights(wb, params, W, sb);
  float *gp = part + (size_t)blockIdx.x * NPAR;
  for (int u = tid; u < NPAR; u += blockDim.x) gp[u] = 0.f;
  for (int u = tid; u < TR * SO; u += blockDim.x) dO[u] = __float2bfloat16_rn(0.f);
  float lsum = 0.f;
  __syncthreads();
  const float scale = 2.f / (float)rows;
  const int64_t tiles = (rows + TR - 1) / TR;
  for (int64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
    const int64_t r0 = tl * TR;
    load_x(feat, r0 + 16 * w, rows, X + 16 * w * S1);
    warp_forward(W, sb, X + 16 * w * S1, H1 + 16 * w * SA, H2 + 16 * w * SA, H3 + 16 * w * SA, out + 16 * w * 2);
    if (lane < 16) {
      const int r = 16 * w + lane;
      const int64_t gr = r0 + r;
      float d0 = 0.f, d1 = 0.f;
      if (gr < rows) {
        d0 = out[r * 2] - target[gr * 2];
        d1 = out[r * 2 + 1] - target[gr * 2 + 1];
      }
      lsum += d0 * d0 + d1 * d1;
      dO[r * SO + 0] = __float2bfloat16_rn(d0 * scale);
      dO[r * SO + 1] = __float2bfloat16_rn(d1 * scale);
    }
    __syncthreads();
    // layer 4: dW4 (2 x 128, warp 0), db4, dZ3
    if (w == 0) {
      float c[16][4];
      zero(c);
      wgemm<16>(c, dO, 1, SO, H3, SA, 1, TR);
      add_acc<16>(gp, OW4, H, c, 0, 2, H);
    }
    if (tid < 2) {
      float s = 0.f;
      for (int r = 0; r < TR; ++r) s += __bfloat162float(dO[r * SO + tid]);
      gp[OB4 + tid] += s;
    }
    back_layer(dO + 16 * w * SO, SO, 16, W + BW4, H3 + 16 * w * SA, Za + 16 * w * SA);
    __syncthreads();
    // layer 3: dW3 += Za' H2, db3, dZ2 -> Zb
    weight_grad<16>(gp, OW3, H, Za, H2, SA, H);
    bias_grad(gp, OB3, Za);
    back_layer(Za + 16 * w * SA, SA, H, W + BW3, H2 + 16 * w * SA, Zb + 16 * w * SA);
    __syncthreads();
    // layer 2: dW2 += Zb' H1, db2, dZ1 -> Za
    weight_grad<16>(gp, OW2, H, Zb, H1, SA, H);
    bias_grad(gp, OB2, Zb);
    __syncthreads();
    back_layer(Zb + 16 * w * SA, SA, H, W + BW2, H1 + 16 * w * SA, Za + 16 * w * SA);
    __syncthreads();
    // layer 1: dW1 += Za' X (25 input columns), db1
    weight_grad<4>(gp, OW1, F, Za, X, S1, F);
    bias_grad(gp, OB1, Za);
    __syncthreads();
  }
  lsum = warp_sum(lsum);
  __shared__ float ls[4];
  if (lane == 0) ls[w] = lsum;
  __syncthreads();
  if (tid == 0) loss_part[blockIdx.x] = ls[0] + ls[1] + ls[2] + ls[3];
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
// x += clip(du e_r + dv e_t, 0.25) per circle; the old coordinates go to backup
__global__ void apply_kernel(StandaloneParams P, const float *__restrict__ dout, float2 *backup) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const float2 x = P.x32[gi];
  backup[gi] = x;
  const float2 er = frame_er(x);
  const float du = dout[2 * gi], dv = dout[2 * gi + 1];
  float dx = du * er.x - dv * er.y, dy = du * er.y + dv * er.x;
  const float nrm = sqrtf(dx * dx + dy * dy);
  if (nrm > 0.25f) { dx *= 0.25f / nrm; dy *= 0.25f / nrm; }
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
                        cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e) return e;
    attr = true;
  }
  if (rows <= 0) return cudaSuccess;
  const int64_t tiles = (rows + 15) / 16;
  const int grid = (int)std::min<int64_t>((tiles + 3) / 4, (int64_t)sms * 2);
  forward_kernel<<<grid, 128, kFwdSmem, s>>>(wb, params, feat, rows, out);
  return cudaGetLastError();
}

int mlp_train_blocks(int sms) { return sms; }

cudaError_t mlp_grad(const bf16 *wb, const float *params, const float *feat, const float *target, int64_t rows,
                     float *part, float *lpart, float *grad, float *loss, int sms, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e) return e;
    attr = true;
  }
  const int nb = mlp_train_blocks(sms);
  train_kernel<<<nb, 128, kTrainSmem, s>>>(wb, params, feat, target, rows, part, lpart);
  grad_reduce_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(part, nb, grad, lpart, rows, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, float *m, float *v, const float *grad, bf16 *wb, float lr, int step,
                     cudaStream_t s) {
  const float b1c = 1.f - powf(0.9f, (float)step), b2c = 1.f - powf(0.999f, (float)step);
  adam_kernel<<<nblk(NPAR, 256), 256, 0, s>>>(params, m, v, grad, wb, lr, b1c, b2c);
  return cudaGetLastError();
}

cudaError_t mlp_apply(const StandaloneParams &p, const float *dout, float2 *backup, cudaStream_t s) {
  if (p.total > 0) apply_kernel<<<nblk(p.total, 256), 256, 0, s>>>(p, dout, backup);
  return cudaGetLastError();
}

cudaError_t mlp_revert(const StandaloneParams &p, const float2 *backup, const double *Eb, const double *Ea,
                       int32_t *accepted, cudaStream_t s) {
  if (p.total > 0) revert_kernel<<<nblk(p.total, 256), 256, 0, s>>>(p, backup, Eb, Ea, accepted);
  return cudaGetLastError();
}

}  // namespace pecc
