// pecc_dev.cuh -- device building blocks shared by the library's kernels.
//
// Elastic model of Sec. 3.2 (Eq. 3, Eq. 5), neighbor sets of Sec. 4.3, and
// the arithmetic forms the descent runs in:
//   Arith32  binary32 coordinates, pair math, gradient, energy accumulation
//   Arith64  binary64 everywhere (the plain FP64 form)
//   ArithMix binary64 coordinates, pair differences and the near-contact
//            quantities 4 - l^2 (two fused multiply-adds) and r^2 - (R-1)^2
//            (exact by Sterbenz' lemma where it cancels); binary32 for
//            everything that only needs relative accuracy (the overlap depth
//            from them, unit vectors, gradient, quasi-Newton vectors), binary64
//            energy sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pecc {

constexpr int kMaxSlots = 11;        // m + 1 physical secant slots, m <= 10
constexpr int kBasis = 2 * kMaxSlots + 1;  // S slots, Y slots, g
constexpr int kMaxK = 64;            // batches per instance
constexpr int kMetaInts = 24;        // per batch: count, stage, ring[kMaxSlots], ...
constexpr int kMaxThreads = 1024;

// ---------------------------------------------------------------- layout ----
struct InstDesc {
  int32_t n, k, ncx, cap;   // circles, batches, cells per side, CSR capacity per buffer
  int32_t big, pad_;        // 1: descended by the whole GPU (pecc_grid.cu), not by one block
  int64_t off;              // first circle (positions, per-circle scratch)
  int64_t rp_off;           // 2 * (n + 1) row pointers (two CSR buffers)
  int64_t col_off;          // 2 * cap column entries (descent lists)
  int64_t col_s_off;        // cap column entries (standalone lists; row pointers at off + index)
  int64_t cell_off;         // 2 * ncell + 2 cell counters
  int64_t gram_off;         // k * kBasis * kBasis Gram entries
  int64_t meta_off;         // k * kMetaInts ring metadata
  double R, inv_cs;
  float inv_f;              // binary32 grid of the FP32 descent: 1 / side, side >= l_cut (1 + 2^-10)
  int32_t ncx_f;            // its cells per side (<= ncx)
};

struct InstOut {
  int32_t iters, status, builds, changes, trials, resets, stalls, polished;
  int32_t iters32, status32, trials32, cur;
  double E, E32, max_overlap, pad;
};

// ------------------------------------------------------------ vec types ----
template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };
template <typename T> using v2 = typename V2<T>::type;

template <typename T> __device__ __forceinline__ v2<T> mk2(T a, T b) { v2<T> r; r.x = a; r.y = b; return r; }

// ---------------------------------------------------------------- philox ---
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    uint4 n;
    n.x = hi1 ^ c.y ^ k.x;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k.y;
    n.w = lo0;
    c = n;
  }
  return c;
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
  return __dmul_rn((double)(w >> 11), 1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------- cells ----
__device__ __forceinline__ int cell_coord(double v, double R, double inv, int nc) {
  double f = __dmul_rn(__dadd_rn(v, R), inv);
  if (!(f >= 0.0)) return 0;
  if (f >= (double)nc) return nc - 1;
  return (int)f;
}

template <typename T>
__device__ __forceinline__ uint32_t cell_key(v2<T> p, double R, double inv, int nc) {
  int cx = cell_coord((double)p.x, R, inv, nc);
  int cy = cell_coord((double)p.y, R, inv, nc);
  return (uint32_t)cy * (uint32_t)nc + (uint32_t)cx;
}

// Neighbor predicate of Sec. 4.3: dx*dx + dy*dy < l_cut^2 with every operation
// correctly rounded (no contraction), in the coordinates' own precision.
__device__ __forceinline__ bool nbr_pred(float2 a, float2 b, float lc2) {
  float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y);
  float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
  return s < lc2;
}
__device__ __forceinline__ bool nbr_pred(double2 a, double2 b, double lc2) {
  double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
  double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return s < lc2;
}

// ------------------------------------------------------------ reductions ---
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV values per thread; every thread receives the totals in out[].
// scratch: at least (blockDim/32) * NV elements of T in shared memory.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T *scratch, T *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    T s = warp_sum(v[q]);
    if (lane == 0) scratch[w * NV + q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NV; q += blockDim.x) {
    T s = T(0);
    for (int u = 0; u < nw; ++u) s += scratch[u * NV + q];
    out[q] = s;
  }
  __syncthreads();
}

// Reduce-scatter of NV values over the 32 lanes of a warp (NV a multiple of 32): after the
// call, lane L holds in v[0 .. NV/32) the warp totals of the values with indices
// (NV/32) * L + j.  Takes NV - NV/32 shuffles instead of 5 NV for NV separate reductions.
template <typename T, int NV>
__device__ __forceinline__ void warp_reduce_scatter(T (&v)[NV]) {
  static_assert(NV % 32 == 0, "NV must be a multiple of 32");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, len = NV; o > 0; o >>= 1, len >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < len / 2; ++j) {
      T keep = hi ? v[j + len / 2] : v[j];
      T send = hi ? v[j] : v[j + len / 2];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// Inclusive prefix sum of a[0..len) in place (int32), whole block; copy (may be null) receives the
// same sums.
__device__ inline void block_scan_inplace(int32_t *a, int len, int32_t *sh /*>=33 ints*/, int32_t *copy = nullptr) {
  const int T = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = T >> 5;
  int ch = (len + T - 1) / T;
  int lo = min(len, t * ch), hi = min(len, lo + ch);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t v = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) sh[lane] = v;
  }
  __syncthreads();
  int32_t run = incl - s + (w > 0 ? sh[w - 1] : 0);
  if (copy)
    for (int i = lo; i < hi; ++i) { run += a[i]; a[i] = run; copy[i] = run; }
  else
    for (int i = lo; i < hi; ++i) { run += a[i]; a[i] = run; }
  __syncthreads();
}

// ------------------------------------------------------- neighbor build ----
// Cell grid of one instance.  Binary64 keys use the grid of the host (side l_cut (1 + 2^-20));
// the binary32 descent uses its own grid with side l_cut (1 + 2^-10), a margin far above the
// rounding of (x + R) / side in binary32, so that circles closer than l_cut are never two
// cells apart.  Either grid only accelerates the search: the set Gamma(i) is fixed by the
// predicate alone.
struct CellGrid {
  double R, inv;
  float Rf, invf;
  int nc;
  bool f32;
};

template <typename T>
__device__ __forceinline__ uint32_t grid_key(v2<T> p, const CellGrid &G) {
  if (G.f32) {
    float fx = ((float)p.x + G.Rf) * G.invf, fy = ((float)p.y + G.Rf) * G.invf;
    int cx = !(fx >= 0.f) ? 0 : (fx >= (float)G.nc ? G.nc - 1 : (int)fx);
    int cy = !(fy >= 0.f) ? 0 : (fy >= (float)G.nc ? G.nc - 1 : (int)fy);
    return (uint32_t)cy * (uint32_t)G.nc + (uint32_t)cx;
  }
  return cell_key<T>(p, G.R, G.inv, G.nc);
}

// 32-bit integer finaliser (xor-shift-multiply); a pair's digest term.  The digest only
// decides ANM's deferral length, never which list is used, so a collision costs nothing but
// a schedule change.
__device__ __forceinline__ unsigned long long mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du;
  x ^= x >> 15; x *= 0x846ca68bu;
  x ^= x >> 16;
  return (unsigned long long)x;
}

// Cell binning and stable key sort, then CSR rows over the 3x3 cells.  x: n positions of
// one instance; lists go to rp[0..n], col[0..cap).  cells: 2 * nc^2 + 2 int32 of scratch;
// ckey/corder: n each; xs: n positions of scratch (the coordinates in cell order, so that
// the three cells of a row of the 3x3 block are one contiguous range).  All pointers may
// be shared or global memory.  sort_rows: rows ascending in j (else in cell-scan order,
// still deterministic).  Returns the number of entries (block-uniform); > cap means
// overflow and the rows are then not written.  hash (shared, may be null) receives an
// order-independent 64-bit digest of the pair set, used to tell Gamma' from Gamma.
// Cell binning and stable key sort of one instance (the first half of a list build): ckey[i]
// = cell of circle i, corder = circles sorted by (cell, index), cells[0..ncell] = cell starts
// (cells[ncell + 1 ..] is scratch), xs[q] = coordinates of corder[q].
template <typename T>
__device__ void cta_cell_sort(const v2<T> *__restrict__ x, int n, const CellGrid &G, uint32_t *ckey,
                              int32_t *corder, int32_t *cells, v2<T> *xs, int32_t *sh) {
  const int T_ = blockDim.x, t = threadIdx.x;
  const int ncell = G.nc * G.nc;
  int32_t *cstart = cells;              // ncell + 1
  int32_t *cfill = cells + ncell + 1;   // ncell
  for (int c = t; c <= ncell; c += T_) cstart[c] = 0;
  __syncthreads();
  for (int i = t; i < n; i += T_) {
    uint32_t key = grid_key<T>(x[i], G);
    ckey[i] = key;
    atomicAdd(&cstart[key + 1], 1);
  }
  __syncthreads();
  // the scan leaves the cell starts in cstart[1..] and, shifted by one, the fill cursors in cfill
  // (cfill[c] = cstart[c]: cell 0 starts at 0)
  if (t == 0) cfill[0] = 0;
  block_scan_inplace(cstart + 1, ncell, sh, cfill + 1);
  for (int i = t; i < n; i += T_) {
    int p = atomicAdd(&cfill[ckey[i]], 1);
    corder[p] = i;
  }
  __syncthreads();
  // stable order: sort every cell's members by index, then their coordinates in that order
  for (int c = t; c < ncell; c += T_) {
    int lo = cstart[c], hi = cstart[c + 1];
    for (int a = lo + 1; a < hi; ++a) {
      int v = corder[a], b = a - 1;
      while (b >= lo && corder[b] > v) { corder[b + 1] = corder[b]; --b; }
      corder[b + 1] = v;
    }
    for (int a = lo; a < hi; ++a) xs[a] = x[corder[a]];
  }
  __syncthreads();
}

template <typename T, typename IdxT>
__device__ int cta_build_neighbors(const v2<T> *__restrict__ x, int n, const CellGrid &G, T lc2,
                                   uint32_t *ckey, int32_t *corder, int32_t *cells, v2<T> *xs, int32_t *rp,
                                   IdxT *col, int cap, int32_t *sh, unsigned long long *hash, bool sort_rows) {
  const int T_ = blockDim.x, t = threadIdx.x;
  const int nc = G.nc;
  int32_t *cstart = cells;
  if (t == 0 && hash) *hash = 0ull;
  cta_cell_sort<T>(x, n, G, ckey, corder, cells, xs, sh);
  if (t == 0) rp[0] = 0;
  __syncthreads();
  // count: circles visited in cell order, candidates as three contiguous row ranges
  for (int q0 = t; q0 < n; q0 += T_) {
    const int i = corder[q0];
    const v2<T> xi = xs[q0];
    const uint32_t key = ckey[i];
    const int cx = (int)(key % (uint32_t)nc), cy = (int)(key / (uint32_t)nc);
    const int bx0 = max(cx - 1, 0), bx1 = min(cx + 1, nc - 1);
    int cntn = 0;
    for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by) {
      const int lo = cstart[by * nc + bx0], hi = cstart[by * nc + bx1 + 1];
      for (int qq = lo; qq < hi; ++qq) cntn += nbr_pred(xi, xs[qq], lc2) && qq != q0;
    }
    rp[i + 1] = cntn;
  }
  __syncthreads();
  block_scan_inplace(rp + 1, n, sh);
  const int total = rp[n];
  if (total <= cap) {
    unsigned long long h = 0ull;
    for (int q0 = t; q0 < n; q0 += T_) {
      const int i = corder[q0];
      const v2<T> xi = xs[q0];
      const uint32_t key = ckey[i];
      const int cx = (int)(key % (uint32_t)nc), cy = (int)(key / (uint32_t)nc);
      const int bx0 = max(cx - 1, 0), bx1 = min(cx + 1, nc - 1);
      int w = rp[i];
      const int first = w;
      for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by) {
        const int lo = cstart[by * nc + bx0], hi = cstart[by * nc + bx1 + 1];
        for (int qq = lo; qq < hi; ++qq) {
          if (nbr_pred(xi, xs[qq], lc2) && qq != q0) {
            const int j = corder[qq];
            col[w++] = (IdxT)j;
            if (hash) h += mix32((uint32_t)i * 0x9E3779B1u ^ (uint32_t)j);
          }
        }
      }
      if (sort_rows) {
        for (int a = first + 1; a < w; ++a) {
          IdxT v = col[a];
          int b = a - 1;
          while (b >= first && col[b] > v) { col[b + 1] = col[b]; --b; }
          col[b + 1] = v;
        }
      }
    }
    if (hash) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
      if ((t & 31) == 0) atomicAdd(hash, h);
    }
  }
  __syncthreads();
  return total;
}

// ------------------------------------------------------------- partition ---
// Order-preserving map of a double onto uint64 (for sorting keys of either sign).
__device__ __forceinline__ uint64_t sortable(double v) {
  uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Partition key of Sec. 4.1 with correctly rounded operations: 0 sector (a pseudo-angle,
// strictly increasing in the polar angle on [0, 2 pi)), 1 annulus (radius), 2 fence (x).
__device__ __forceinline__ double part_key(double x, double y, int mode) {
  if (mode == 1) return __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  if (mode == 2) return x;
  double s = __dadd_rn(fabs(x), fabs(y));
  if (s == 0.0) return 0.0;
  double t = __ddiv_rn(x, s);
  return (y >= 0.0) ? __dsub_rn(1.0, t) : __dadd_rn(3.0, t);
}

// Key of the random partition of Sec. 4.1 (mode 3): 53 bits of Philox4x32-10 counter
// (i, 0, q, 3 * 2^30) under the partition seed; the order by (key, index) is a uniform permutation.
__device__ __forceinline__ double random_part_key(uint64_t seed, int i, int q) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, (uint32_t)q, 0xC0000000u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return u53(w.x, w.y);
}

// ------------------------------------------------------- pair arithmetic ---
// pair(): for circles a (the row owner) and b, returns the overlap depth d >= 0
// (0 when l >= 2) and the gradient contribution to a: -2 d (a - b) / l.
// A coincident pair contributes d = 2 and no gradient.
struct Arith32 {
  using pos_t = float;
  using vec_t = float;
  using acc_t = float;
  static constexpr int kId = 1;
  // Without branches: every lane of a warp takes the same instructions whether its pair is in
  // contact or not (a list row holds both kinds), and the selects give the values of the case split.
  __device__ static __forceinline__ acc_t pair(float2 a, float2 b, float &fx, float &fy) {
    float dx = a.x - b.x, dy = a.y - b.y;
    float s = dx * dx + dy * dy;
    const bool act = s < 4.f, pos = s > 0.f, ap = act && pos;
    float rl = rsqrtf(pos ? s : 1.f);
    float d = 2.f - s * rl;
    float c = -2.f * d * rl;
    fx = ap ? c * dx : 0.f;
    fy = ap ? c * dy : 0.f;
    return act ? (pos ? fmaxf(d, 0.f) : 2.f) : 0.f;
  }
  // The same values with the arithmetic of pairs beyond contact skipped by a branch: the standalone
  // energy + gradient kernel's rows at converged layouts hold many such pairs, and there the skip
  // saves more than keeping the lanes together (3 % on the batch's final layouts).
  __device__ static __forceinline__ acc_t pair_skip(float2 a, float2 b, float &fx, float &fy) {
    float dx = a.x - b.x, dy = a.y - b.y;
    float s = dx * dx + dy * dy;
    fx = 0.f; fy = 0.f;
    if (!(s < 4.f)) return 0.f;
    if (s > 0.f) {
      float rl = rsqrtf(s);
      float d = 2.f - s * rl;
      float c = -2.f * d * rl;
      fx = c * dx; fy = c * dy;
      return fmaxf(d, 0.f);
    }
    return 2.f;
  }
  // container term: depth d_i0 and gradient 2 d_i0 c_i / |c_i|
  __device__ static __forceinline__ acc_t wall(float2 a, float R, float Rm1sq, float &fx, float &fy) {
    float r2 = a.x * a.x + a.y * a.y;
    float r = sqrtf(r2);
    float d = r + 1.f - R;
    fx = 0.f; fy = 0.f;
    if (!(d > 0.f)) return 0.f;
    if (r > 0.f) { float c = 2.f * d / r; fx = c * a.x; fy = c * a.y; }
    return d;
  }
};

__device__ __forceinline__ double rsqrt_d(double s) {
  // binary32 estimate refined by two Newton steps in binary64 (s >= 1e-30)
  double y = (double)rsqrtf((float)s);
  double h = 0.5 * s;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

struct Arith64 {
  using pos_t = double;
  using vec_t = double;
  using acc_t = double;
  static constexpr int kId = 0;
  __device__ static __forceinline__ acc_t pair(double2 a, double2 b, double &fx, double &fy) {
    double dx = a.x - b.x, dy = a.y - b.y;
    double s = fma(dx, dx, dy * dy);
    fx = 0.0; fy = 0.0;
    if (!(s < 4.0)) return 0.0;
    if (s > 1e-30) {
      double rl = rsqrt_d(s);
      double d = 2.0 - s * rl;
      double c = -2.0 * d * rl;
      fx = c * dx; fy = c * dy;
      return d > 0.0 ? d : 0.0;
    }
    if (s > 0.0) {
      double l = sqrt(s);
      double c = -2.0 * (2.0 - l) / l;
      fx = c * dx; fy = c * dy;
      return 2.0 - l;
    }
    return 2.0;
  }
  // pair() already skips the pairs beyond contact
  __device__ static __forceinline__ acc_t pair_skip(double2 a, double2 b, double &fx, double &fy) {
    return pair(a, b, fx, fy);
  }
  // Rm1sq = (R - 1)^2 when R >= 1, else -1 (every circle then touches the wall)
  __device__ static __forceinline__ acc_t wall(double2 a, double R, double Rm1sq, double &fx, double &fy) {
    double r2 = fma(a.x, a.x, a.y * a.y);
    fx = 0.0; fy = 0.0;
    if (!(r2 > Rm1sq)) return 0.0;  // |c| <= R - 1: no contact
    if (r2 <= 1e-30) { double d = sqrt(r2) + 1.0 - R; return d > 0.0 ? d : 0.0; }
    double rl = rsqrt_d(r2);
    double r = r2 * rl;
    double d = r + 1.0 - R;
    if (!(d > 0.0)) return 0.0;
    double c = 2.0 * d * rl;
    fx = c * a.x; fy = c * a.y;
    return d;
  }
};

struct ArithMix {
  using pos_t = double;
  using vec_t = float;
  using acc_t = double;
  static constexpr int kId = 2;
  // 4 - l^2 = 4 - dy^2 - dx^2 by two fused multiply-adds (one rounding of size ulp64(4) / 2 at
  // most, then the exact cancellation near contact and one rounding of the small result); its
  // sign is the contact test, and everything after it is binary32.
  __device__ static __forceinline__ float pair(double2 a, double2 b, float &fx, float &fy) {
    const double dx = a.x - b.x, dy = a.y - b.y;
    const float e = (float)fma(-dx, dx, fma(-dy, dy, 4.0));
    fx = 0.f; fy = 0.f;
    if (!(e > 0.f)) return 0.f;
    const float dxf = (float)dx, dyf = (float)dy;
    const float s = fmaf(dxf, dxf, dyf * dyf);
    if (s > 1e-30f) {
      const float rl = rsqrtf(s);
      const float l = s * rl;
      const float d = e / (2.f + l);    // 2 - l = (4 - l^2) / (2 + l)
      const float c = -2.f * d * rl;
      fx = c * dxf; fy = c * dyf;
      return d;
    }
    return 2.f;
  }
  // pair() already skips the pairs beyond contact
  __device__ static __forceinline__ float pair_skip(double2 a, double2 b, float &fx, float &fy) {
    return pair(a, b, fx, fy);
  }
  __device__ static __forceinline__ acc_t wall(double2 a, double R, double Rm1sq, float &fx, float &fy) {
    double r2 = fma(a.x, a.x, a.y * a.y);
    fx = 0.f; fy = 0.f;
    if (!(r2 > Rm1sq)) return 0.0;
    if (Rm1sq < 0.0 || r2 <= 1e-30) {   // degenerate container R < 1, or a centred circle
      double r = sqrt(r2), d = r + 1.0 - R;
      if (r > 0.0) { float c = (float)(2.0 * d / r); fx = c * (float)a.x; fy = c * (float)a.y; }
      return d > 0.0 ? d : 0.0;
    }
    float e = (float)(r2 - Rm1sq);      // |c|^2 - (R-1)^2, exact near contact
    float r = sqrtf((float)r2);
    float d = e / (r + (float)(R - 1.0));  // |c| - (R - 1)
    float c = 2.f * d / r;
    fx = c * (float)a.x; fy = c * (float)a.y;
    return (double)d;
  }
};

// Exact container depth with correctly rounded operations (feasibility check).
__device__ __forceinline__ double wall_depth_exact(double2 a, double R) {
  double r = __dsqrt_rn(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)));
  double d = __dsub_rn(__dadd_rn(r, 1.0), R);
  return d > 0.0 ? d : 0.0;
}
__device__ __forceinline__ double pair_depth_exact(double2 a, double2 b) {
  double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
  double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return __dsub_rn(2.0, __dsqrt_rn(s));
}

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace pecc
