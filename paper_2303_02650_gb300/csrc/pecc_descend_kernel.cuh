// pecc_descend_kernel.cuh -- persistent descent kernel: Algorithm GBO (Sec. 4.1) with ANM (Sec. 4.3).
//
// One thread block owns one instance at a time and pops the next instance from
// a device work queue when it is done.  Inside the block:
//   * partition: circles ranked by the partition key (sector: pseudo-angle of
//     the polar angle; annulus: radius; fence: x), ties by index, then cut into
//     k contiguous batches of floor(n/k) or ceil(n/k) circles (Sec. 4.1).  The
//     instance is renumbered in that order, so batch p is a contiguous range of
//     every per-circle array and "merge" is a scatter at the end.
//   * neighbor lists: cell binning + stable key sort + 3x3-cell CSR build, in the
//     block (cta_build_neighbors).  Rebuilt by ANM after every sweep (Algorithm
//     ANM: Gamma' replaces Gamma, and whether it differs -- compared through an
//     order-independent 64-bit digest of the pair set -- decides the deferral
//     length) and before a batch step whenever twice the largest displacement since
//     the last build plus the step cap could exceed l_cut - 2 (Verlet rule).
//   * per batch step (Eq. 8): the batch energy of Eq. 7 and its gradient, the
//     quasi-Newton direction -H g of Eq. 10 / Eq. 11 with m secant pairs, a
//     backtracking line search in place of the argmin of Eq. 9, and a secant
//     pair push when the curvature condition holds.
//
// The instance's working set (coordinates, gradients, direction, neighbor lists,
// cell scratch, Gram matrices, and last the secant pairs) is carved out of dynamic shared
// memory as far as it fits, the rest falls back to global memory; with thousands of instances
// in flight the secant pairs stay in global memory (read coalesced, L2-resident), a block alone
// on its SM holds them on chip.
//
// The direction is computed in "vector-free" form (Chen, Wang, Zhou, Burges,
// "Large-scale L-BFGS using MapReduce", NIPS 2014): the two-loop recursion is
// run on the Gram matrix of the basis {s_a, y_a, g} by one warp, and the direction
// is assembled as one linear combination.  In exact arithmetic this is the
// two-loop recursion; it replaces 2m dependent block-wide dot products by one
// batched reduction per step.
#pragma once
#include <cfloat>

#include "pecc_internal.h"

namespace pecc {

namespace {

constexpr int KS = kMaxSlots;     // basis index of Y slot a is KS + a
constexpr int GI = 2 * kMaxSlots; // basis index of g
// The dots of the first reduction of a batch step come in chunks of 32 values, one chunk per four
// physical slots a: in chunk a / 4, from 6 (a % 4): g's_a, g'y_a, s's_a, s'y_a, y's_a, y'y_a, where
// (s, y) is the pending pair; chunk 0 also carries g'g, s's, s'y and y'y at 24..27.
constexpr int kSlotsPerChunk = 4;
constexpr int kChunks = (kMaxSlots + kSlotsPerChunk - 1) / kSlotsPerChunk;
constexpr int kPA = 32 * kChunks;  // per-warp partial values of the first reduction
constexpr int PA_GG = 24, PA_SS = 25, PA_SY = 26, PA_YY = 27;
__device__ __forceinline__ int pa_idx(int a, int kind) { return 32 * (a >> 2) + 6 * (a & 3) + kind; }
constexpr int kRingInts = kMaxSlots + 3;  // count, stage, ring[kMaxSlots], pending

__device__ __forceinline__ uint64_t sortable(double v) {
  uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Partition key of Sec. 4.1 with correctly rounded operations.
__device__ __forceinline__ double part_key(double x, double y, int mode) {
  if (mode == 1) return __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  if (mode == 2) return x;
  double s = __dadd_rn(fabs(x), fabs(y));
  if (s == 0.0) return 0.0;
  double t = __ddiv_rn(x, s);
  return (y >= 0.0) ? __dsub_rn(1.0, t) : __dadd_rn(3.0, t);
}

// W: warps per block, at most
template <class A, int W> struct Smem {
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  acc_t rs[2][W];              // single-barrier reductions: per-warp sums, two alternating buffers
  vec_t rm[2][W];              // and per-warp maxima
  vec_t ob[kPA];               // totals of the first reduction of a batch step (written by warp 0)
  acc_t eA;                    // batch energy of that reduction
  vec_t coef[kBasis];
  unsigned long long hash;
  unsigned used;               // physical slots in the current batch's ring (bit mask)
  int32_t sh[40];
  int q;
  int flag;
};

// Block reduction of one sum and one maximum with a single barrier.  Every warp leaves its results
// in buffer `buf`, and every thread then combines them itself; consecutive reductions alternate
// buffers, so a fast thread's writes for the next reduction cannot overtake a slow thread's reads
// of this one (a barrier of the reduction in between separates them).
template <class A, int W>
__device__ __forceinline__ void reduce_sm(Smem<A, W> &S, int &buf, typename A::acc_t &a, typename A::vec_t &m) {
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const acc_t ws = warp_sum(a);
  const vec_t wm = warp_max(m);
  if (lane == 0) { S.rs[buf][w] = ws; S.rm[buf][w] = wm; }
  __syncthreads();
  acc_t sa = S.rs[buf][0];
  vec_t sm = S.rm[buf][0];
  // the loads of every warp's partial are independent: unrolled to the block's warp bound so that
  // they are all in flight, the additions keep the warp order
#pragma unroll
  for (int u = 1; u < W; ++u)
    if (u < nw) { sa += S.rs[buf][u]; sm = max(sm, S.rm[buf][u]); }
  a = sa;
  m = sm;
  buf ^= 1;
}

// Forces on circle pos from the entries col[t0 .. t1) of its row, added to (gx, gy), and its share
// of the batch energy added to ei: the pairs with a circle outside the batch [b, e) or inside it
// with a smaller index.  Two entries per step, so that the loads of both are in flight together;
// the sums take the entries in row order, the values of one entry per step.
template <class A, typename PP>
__device__ __forceinline__ void row_terms(const PP xi, const uint16_t *__restrict__ col, int t0, int t1,
                                          const PP *__restrict__ xw, int b, int e, int pos,
                                          typename A::vec_t &gx, typename A::vec_t &gy, typename A::acc_t &ei) {
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  for (int t = t0; t < t1; t += 2) {
    const bool two = t + 1 < t1;
    const int j1 = col[t];
    const int j2 = two ? (int)col[t + 1] : j1;
    const PP x1 = xw[j1], x2 = xw[j2];
    vec_t fx, fy;
    const auto d1 = A::pair(xi, x1, fx, fy);
    gx += fx; gy += fy;
    if (j1 < b || j1 >= e || j1 < pos) ei += (acc_t)d1 * (acc_t)d1;
    if (two) {
      const auto d2 = A::pair(xi, x2, fx, fy);
      gx += fx; gy += fy;
      if (j2 < b || j2 >= e || j2 < pos) ei += (acc_t)d2 * (acc_t)d2;
    }
  }
}

// Bump allocator over dynamic shared memory; returns the fallback when the request does not fit.
struct Carve {
  unsigned char *base;
  size_t cap, used;
  template <typename T> __device__ T *take(size_t count, T *fallback) {
    size_t b = (count * sizeof(T) + 15) & ~size_t(15);
    if (used + b <= cap) {
      T *p = (T *)(base + used);
      used += b;
      return p;
    }
    return fallback;
  }
};


// One instance q of the descent, run by the whole block (the body of the persistent loops below).
// W: warps per block, at most.
template <class A, int W>
__device__ __forceinline__ void descend_instance(const DescendParams &P, Smem<A, W> &S, unsigned char *dsm, int q) {
  using pos_t = typename A::pos_t;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  using sc_t = acc_t;  // per-step scalars in the arithmetic's own precision
  using PP = v2<pos_t>;
  using VV = v2<vec_t>;
  const sc_t c1 = (sc_t)P.c1, step_max = (sc_t)P.step_max, two_skin = (sc_t)(2.0 * P.rebuild_disp);
  const sc_t gsum_tol = (sc_t)P.gsum_tol, curv_eps = (sc_t)P.curv_eps;
  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int mm = P.m + 1;  // physical slots

  const InstDesc D = P.desc[q];
  if (D.big) return;  // descended by the whole GPU after this launch (uniform across the block)
  InstOut *O = P.out + q;
  const int n = D.n;
  const acc_t R = (acc_t)D.R;
  const acc_t Rm1sq = (acc_t)((D.R >= 1.0) ? (D.R - 1.0) * (D.R - 1.0) : -1.0);

  // ---- phase entry: the polish runs only on instances the FP32 descent left near zero energy
  if (A::kId == 2) {
    bool skip = !(O->E32 <= P.polish_gate) || O->status32 >= 4;
    if (skip) {
      for (int i = tid; i < n; i += T) {
        float2 v = P.x32[D.off + i];
        P.x64[D.off + i] = make_double2((double)v.x, (double)v.y);
      }
      if (tid == 0) {
        O->iters = O->iters32; O->status = O->status32; O->E = O->E32; O->polished = 0;
      }
      __syncthreads();
      return;
    }
  }
  if (n == 0) {
    if (tid == 0) {
      O->iters = 0; O->status = 0; O->E = 0.0;
      if (A::kId == 1) { O->iters32 = 0; O->status32 = 0; O->E32 = 0.0; O->trials32 = 0; }
    }
    __syncthreads();
    return;
  }
  const int k = (P.k_override > 0) ? min(P.k_override, D.k) : D.k;

  // ---- working set: shared memory first, global scratch as the fallback.  A per-circle fallback
  // starts at the instance's offset counted in double2 (16 B) whatever the arithmetic, so the FP32
  // phase of one instance and the polish of another, running at the same time in the fused
  // kernel, never share bytes.  The per-warp partials
  // of the first reduction and the batch rings have no fallback (the launch plan reserves them);
  // then the Gram matrices (the two-loop's dependent chain), the arrays every pass touches, and
  // last the scratch of the list builds.
  const int nw = T >> 5;
  Carve cv{dsm, P.smem_bytes, 0};
  vec_t *pa = cv.take<vec_t>((size_t)nw * kPA, (vec_t *)nullptr);
  int *rings = cv.take<int>((size_t)k * kRingInts, (int *)nullptr);
  if (pa == nullptr || rings == nullptr) {  // a launch plan too small for this instance
    if (tid == 0) { O->iters = 0; O->status = 4; O->E = 0.0; if (A::kId == 1) { O->iters32 = 0; O->status32 = 4; } }
    __syncthreads();
    return;
  }
  vec_t *gram = cv.take<vec_t>((size_t)k * kBasis * kBasis, (vec_t *)P.gram + D.gram_off);
  PP *xw = cv.take<PP>(n, (PP *)((double2 *)P.xw + D.off));
  int32_t *rp = cv.take<int32_t>(n + 1, P.rp + D.rp_off);
  // two-level lists: the rows of the filtered lists start where the outer list's rows start and
  // end at re[p]; with one level re = rp + 1 (CSR)
  bool two = P.list_outer > 0.0;
  int32_t *re = two ? cv.take<int32_t>(n, P.rp + D.rp_off + n + 1) : rp + 1;
  // neighbor indices are 16-bit inside the descent (instances of at most 65535 circles)
  const int cap_s = min(D.cap, 8 * n + 64);  // about 5 neighbors per circle in practice
  uint16_t *col_s = cv.take<uint16_t>(cap_s, (uint16_t *)nullptr);
  uint16_t *const col_g = (uint16_t *)(P.col + D.col_off);  // 2 cap int32 = 4 cap uint16
  uint16_t *col = col_s ? col_s : col_g;
  int cap = col_s ? cap_s : D.cap;
  VV *g = cv.take<VV>(n, (VV *)((double2 *)P.g + D.off));
  VV *dv = cv.take<VV>(n, (VV *)((double2 *)P.d + D.off));
  VV *gt = cv.take<VV>(n, (VV *)((double2 *)P.gt + D.off));
  PP *xo = cv.take<PP>(n, (PP *)((double2 *)P.xo + D.off));
  PP *xb = cv.take<PP>(n, (PP *)((double2 *)P.xb + D.off));
  const CellGrid G = (A::kId == 1) ? CellGrid{D.R, D.inv_cs, (float)D.R, D.inv_f, D.ncx_f, true}
                                   : CellGrid{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
  // The list builds' scratch lives in arrays that are dead while a build runs: the circles in
  // cell order and their cell keys in the direction (8 n bytes at least), the cell table in the
  // positions at the last build when it fits (they are rewritten right after every build).  The
  // gradient arrays cannot serve: one-batch steps swap g and gt and carry a gradient across the
  // build at the end of a sweep.
  int32_t *corder = (int32_t *)dv;
  uint32_t *ckey = (uint32_t *)dv + n;
  const size_t ncells = 2 * (size_t)G.nc * G.nc + 2;
  int32_t *cells = (ncells * sizeof(int32_t) <= (size_t)n * sizeof(PP)) ? (int32_t *)xb
                                                                       : cv.take<int32_t>(ncells, P.cells + D.cell_off);
  // the secant pairs last: on chip when the block's share holds them (few instances per launch, a
  // block alone on its SM), else in global memory; they carry nothing between descent calls
  VV *Sv = cv.take<VV>((size_t)mm * n, (VV *)P.S + (int64_t)mm * D.off);
  VV *Yv = cv.take<VV>((size_t)mm * n, (VV *)P.Y + (int64_t)mm * D.off);
  // the outer list last: its rows are read once per filtered rebuild
  uint16_t *const colL_g = col_g + 2 * (size_t)D.cap;
  uint16_t *colL_s = nullptr, *colL = nullptr;
  int capL = 0;
  CellGrid GL = G;
  pos_t lc2L = 0;
  if (two) {
    const int capL_s = min(D.cap, kOuterPerCircle * n + 64);
    colL_s = cv.take<uint16_t>(capL_s, (uint16_t *)nullptr);
    colL = colL_s ? colL_s : colL_g;
    capL = colL_s ? capL_s : D.cap;
    const double lb = P.l_cut + P.list_outer;
    double inv;
    int nc;
    host_cell_grid(D.R, lb, n, &inv, &nc);
    if (A::kId == 1) {
      float invf;
      int ncf;
      f32_cell_grid(D.R, lb, n, nc, &invf, &ncf);
      GL = CellGrid{D.R, inv, (float)D.R, invf, ncf, true};
    } else {
      GL = CellGrid{D.R, inv, 0.f, 0.f, nc, false};
    }
    lc2L = (pos_t)(lb * lb);
    if (GL.nc > G.nc) { two = false; re = rp + 1; }  // its cell table must fit the scratch
  }
  int32_t *perm = P.perm + D.off;
  // the partition keys borrow the list storage (8 n bytes) before the first build
  uint64_t *skey = (col_s && (size_t)cap_s * 2 >= (size_t)n * 8) ? (uint64_t *)col_s : P.skey + D.off;
  const pos_t lc2 = (pos_t)(P.l_cut * P.l_cut);

  // ---- 1. partition key and rank (stable by index)
  for (int i = tid; i < n; i += T) {
    double x, y;
    if (A::kId == 0) { double2 v = P.x64[D.off + i]; x = v.x; y = v.y; }
    else { float2 v = P.x32[D.off + i]; x = v.x; y = v.y; }
    skey[i] = sortable(P.partition == 3 ? random_part_key(P.part_seed, i, q) : part_key(x, y, P.partition));
  }
  __syncthreads();
  for (int i = tid; i < n; i += T) {
    uint64_t ki = skey[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      uint64_t kj = skey[j];
      r += (kj < ki) || (kj == ki && j < i);
    }
    perm[r] = i;
  }
  __syncthreads();
  // ---- 2. renumber: working coordinates in partition order
  int bad = 0;
  for (int p = tid; p < n; p += T) {
    int i = perm[p];
    PP v;
    if (A::kId == 0) { double2 u = P.x64[D.off + i]; v.x = (pos_t)u.x; v.y = (pos_t)u.y; }
    else { float2 u = P.x32[D.off + i]; v.x = (pos_t)u.x; v.y = (pos_t)u.y; }
    bad |= !(isfinite((float)v.x) && isfinite((float)v.y));
    xw[p] = v;
  }
  bad |= !(D.R > 0.0 && isfinite(D.R));  // a radius pecc_set_radius could not accept
  bad = __syncthreads_or(bad);

  int status = 3;  // max_iter unless something else ends the run
  bool lists_ok = false;  // the lists and xb hold a complete build
  int iters = 0, builds = 0, changes = 0, trials = 0, resets = 0, stalls = 0;
  int cnt = 0, len = 1;
  unsigned long long hcur = 0ull;  // digest of the current lists
  sc_t Dmax = 0;  // largest displacement since the last build
  acc_t E = 0;
  int rbuf = 0;  // buffer of the next single-barrier reduction (block-uniform)

  // the outer list at the current layout (rows rp, entries colL); the filtered lists take the
  // same room, so they move to global memory with it when it outgrows their share
  auto build_outer = [&]() -> bool {
    int tot = cta_build_neighbors<pos_t, uint16_t>(xw, n, GL, lc2L, ckey, corder, cells, xo, rp, colL, capL, S.sh,
                                                   nullptr, false);
    if (tot > capL && colL_s && colL == colL_s) {
      colL = colL_g;
      capL = D.cap;
      tot = cta_build_neighbors<pos_t, uint16_t>(xw, n, GL, lc2L, ckey, corder, cells, xo, rp, colL, capL, S.sh,
                                                 nullptr, false);
    }
    if (tot > capL) return false;
    if (tot > cap && col_s && col == col_s) {
      col = col_g;
      cap = D.cap;
    }
    return tot <= cap;
  };
  // the lists of Sec. 4.3 from the outer list: the predicate of a cell-grid build on the same
  // coordinates, so the same set (rows in the outer list's order), and the same digest
  auto filter = [&]() {
    if (tid == 0) S.hash = 0ull;
    __syncthreads();
    unsigned long long h = 0ull;
    for (int p = tid; p < n; p += T) {
      const PP xi = xw[p];
      const int t1 = rp[p + 1];
      int w = rp[p];
      for (int t = w; t < t1; t += 8) {
        int jj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) jj[u] = (t + u < t1) ? (int)colL[t + u] : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = jj[u];
          if (j >= 0 && nbr_pred(xi, xw[j], lc2)) {
            col[w++] = (uint16_t)j;
            h += mix32((uint32_t)p * 0x9E3779B1u ^ (uint32_t)j);
          }
        }
      }
      re[p] = w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) atomicAdd(&S.hash, h);
    __syncthreads();
  };
  // bound on the largest displacement since the outer list's build: the sum of the largest
  // displacements between the list builds since then
  sc_t DL = 0;
  bool outer_ok = false;
  const sc_t outer_room = (sc_t)(P.list_outer - 1.0 / 1024.0);
  // one list build into the block's list storage; moves the lists to global memory when they
  // outgrow their shared-memory share; false when even the global capacity is exceeded
  auto build = [&]() -> bool {
    if (two) {
      const sc_t Dnow = DL + Dmax;
      if (outer_ok && sc_t(2) * Dnow < outer_room) {
        DL = Dnow;
      } else {
        outer_ok = build_outer();
        DL = 0;
        if (!outer_ok) { two = false; re = rp + 1; }  // one level from here on
      }
      if (two) { filter(); return true; }
    }
    int tot = cta_build_neighbors<pos_t, uint16_t>(xw, n, G, lc2, ckey, corder, cells, xo, rp, col, cap, S.sh,
                                                   &S.hash, false);
    if (tot > cap && col_s && col == col_s) {
      col = col_g;
      cap = D.cap;
      tot = cta_build_neighbors<pos_t, uint16_t>(xw, n, G, lc2, ckey, corder, cells, xo, rp, col, cap, S.sh,
                                                 &S.hash, false);
    }
    return tot <= cap;
  };
  // ANM step (Algorithm ANM): Gamma' replaces Gamma; equal sets double the deferral length
  auto anm_rebuild = [&]() -> bool {
    if (!build()) { lists_ok = false; return false; }
    ++builds;
    const unsigned long long h = S.hash;
    if (h != hcur) { hcur = h; len = 1; ++changes; }
    else if (len < (1 << 30)) len *= 2;
    cnt = 0;
    for (int p = tid; p < n; p += T) xb[p] = xw[p];
    Dmax = 0;
    __syncthreads();
    return true;
  };
  // full energy (Eq. 5 over the lists: each pair from its larger index)
  auto full_energy = [&]() -> acc_t {
    acc_t a = 0;
    vec_t m = 0;
    for (int p = tid; p < n; p += T) {
      PP xi = xw[p];
      acc_t e = 0;
      vec_t ux = 0, uy = 0;  // unused
      row_terms<A, PP>(xi, col, rp[p], re[p], xw, 0, n, p, ux, uy, e);
      vec_t fx, fy;
      acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
      a += e + d0 * d0;
    }
    reduce_sm<A, W>(S, rbuf, a, m);
    return a;
  };

  if (bad) {
    status = 5;
  } else {
    if (!build()) status = 4;
    else {
      builds = 1;
      lists_ok = true;
      for (int p = tid; p < n; p += T) xb[p] = xw[p];  // the cell table of the build used xb
      hcur = S.hash;
      E = full_energy();
      if (!isfinite(E)) status = 5;
      else if (E <= (acc_t)P.e_tol) status = 0;
    }
  }
  for (int u = tid; u < k * kRingInts; u += T) rings[u] = 0;
  for (int u = tid; u < k * kBasis * kBasis; u += T) gram[u] = vec_t(0);
  __syncthreads();

  const int q_ = n / k, r_ = n % k;
  bool fresh = false;  // k == 1: g / E of the previous accepted trial are current
  int e_at = 0;        // sweep after which E was last evaluated
  acc_t Ewin = E;      // FP32 phase: energy at the start of the stagnation window

  // ---- 3. sweeps
  while (status == 3 && iters < P.max_iter) {
    ++iters;
    sc_t gsum = 0;
    int moved = 0;
    for (int p = 0; p < k && status == 3; ++p) {
      const int b = p * q_ + min(p, r_), e = b + q_ + (p < r_ ? 1 : 0);
      // Verlet guarantee for the coming step
      if (sc_t(2) * Dmax + step_max > two_skin) {
        if (!anm_rebuild()) { status = 4; break; }
        fresh = false;
      }
      int *ring = rings + p * kRingInts;  // [0] count, [1] stage, [2..] slots, [2 + KS] pending
      vec_t *Gm = gram + (size_t)p * kBasis * kBasis;
      const int count0 = ring[0], st = ring[1], pending = ring[2 + kMaxSlots];

      // ---- pass A: batch energy (Eq. 7) and gradient, then the dots of g and of the pair (s, y)
      // written by this batch's previous step with every stored vector (the pair's curvature is
      // tested here).  The pair is staged in the direction and trial-gradient arrays (both free
      // until pass B and pass D), and the dots are taken four slots at a time, each chunk of 32
      // values reduce-scattered over the warp: few live accumulators, many loads in flight.
      if (fresh) { VV *t_ = g; g = gt; gt = t_; }
      acc_t aA = 0;
      vec_t xgg = 0, xss = 0, xsy = 0, xyy = 0;
      for (int pos = b + tid; pos < e; pos += T) {
        PP xi = xw[pos];
        xo[pos] = xi;
        VV gi;
        if (!fresh) {
          vec_t gx = 0, gy = 0;
          acc_t ei = 0;
          row_terms<A, PP>(xi, col, rp[pos], re[pos], xw, b, e, pos, gx, gy, ei);
          vec_t fx, fy;
          acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
          gx += fx; gy += fy;
          aA += ei + d0 * d0;
          gi.x = gx; gi.y = gy;
          g[pos] = gi;
        } else {
          gi = g[pos];
        }
        xgg += gi.x * gi.x + gi.y * gi.y;
        if (pending) {
          const VV sp = Sv[(int64_t)st * n + pos], yp = Yv[(int64_t)st * n + pos];
          dv[pos] = sp;
          gt[pos] = yp;
          xss += sp.x * sp.x + sp.y * sp.y;
          xsy += sp.x * yp.x + sp.y * yp.y;
          xyy += yp.x * yp.x + yp.y * yp.y;
        }
      }
      const int nch = (mm + kSlotsPerChunk - 1) / kSlotsPerChunk;
      for (int c = 0; c < nch; ++c) {
        vec_t v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = 0;
        if (c == 0) { v[PA_GG] = xgg; v[PA_SS] = xss; v[PA_SY] = xsy; v[PA_YY] = xyy; }
        for (int pos = b + tid; pos < e; pos += T) {
          const VV gi = g[pos];
          VV sp{}, yp{};
          if (pending) { sp = dv[pos]; yp = gt[pos]; }
#pragma unroll
          for (int j = 0; j < kSlotsPerChunk; ++j) {
            const int a = c * kSlotsPerChunk + j;
            if (a < mm) {
              const VV s_ = Sv[(int64_t)a * n + pos], y_ = Yv[(int64_t)a * n + pos];
              v[6 * j + 0] += gi.x * s_.x + gi.y * s_.y;
              v[6 * j + 1] += gi.x * y_.x + gi.y * y_.y;
              if (pending) {
                v[6 * j + 2] += sp.x * s_.x + sp.y * s_.y;
                v[6 * j + 3] += sp.x * y_.x + sp.y * y_.y;
                v[6 * j + 4] += yp.x * s_.x + yp.y * s_.y;
                v[6 * j + 5] += yp.x * y_.x + yp.y * y_.y;
              }
            }
          }
        }
        warp_reduce_scatter<vec_t, 32>(v);
        pa[warp * kPA + c * 32 + lane] = v[0];
      }
      {
        const acc_t ws = warp_sum(aA);
        if (lane == 0) S.rs[rbuf][warp] = ws;
      }
      __syncthreads();

      // ---- warp 0: totals, push of the pending pair, two-loop.  The other warps wait at the next
      // barrier; nothing here needs the whole block.
      if (warp == 0) {
        for (int qv = lane; qv < nch * 32; qv += 32) {
          vec_t t = 0;
#pragma unroll
          for (int u = 0; u < W; ++u)
            if (u < nw) t += pa[u * kPA + qv];
          S.ob[qv] = t;
        }
        if (lane == 0) {
          acc_t t = 0;
#pragma unroll
          for (int u = 0; u < W; ++u)
            if (u < nw) t += S.rs[rbuf][u];
          S.eA = t;
        }
        __syncwarp();
        // the pending pair joins the memory when s'y > curv_eps |s| |y| (Gram rows, then the ring)
        if (pending) {
          const vec_t ss = S.ob[PA_SS], sy = S.ob[PA_SY], yy = S.ob[PA_YY];
          const bool push = (sc_t)sy > curv_eps * sqrt((sc_t)ss) * sqrt((sc_t)yy) && P.m > 0;
          if (push) {
            if (lane < count0) {
              const int sl = ring[2 + lane];
              Gm[st * kBasis + sl] = Gm[sl * kBasis + st] = S.ob[pa_idx(sl, 2)];
              Gm[st * kBasis + KS + sl] = Gm[(KS + sl) * kBasis + st] = S.ob[pa_idx(sl, 3)];
              Gm[(KS + st) * kBasis + sl] = Gm[sl * kBasis + KS + st] = S.ob[pa_idx(sl, 4)];
              Gm[(KS + st) * kBasis + KS + sl] = Gm[(KS + sl) * kBasis + KS + st] = S.ob[pa_idx(sl, 5)];
            }
            if (lane == 0) {
              Gm[st * kBasis + st] = ss;
              Gm[st * kBasis + KS + st] = Gm[(KS + st) * kBasis + st] = sy;
              Gm[(KS + st) * kBasis + KS + st] = yy;
            }
          }
          __syncwarp();
          if (push) {
            const int c = ring[0];
            if (c < P.m) {
              // the new stage slot: the lowest physical slot not in the ring once st joins it
              const unsigned inring =
                  __reduce_or_sync(0xffffffffu, lane < c ? (1u << ring[2 + lane]) : 0u) | (1u << st);
              __syncwarp();
              if (lane == 0) {
                ring[2 + c] = st;
                ring[0] = c + 1;
                ring[1] = __ffs(~inring) - 1;
              }
            } else if (lane == 0) {
              int ev = ring[2];
              for (int u = 0; u + 1 < c; ++u) ring[2 + u] = ring[3 + u];
              ring[2 + c - 1] = st;
              ring[1] = ev;
            }
          }
          if (lane == 0) ring[2 + kMaxSlots] = 0;
          __syncwarp();
        }
        const int count = ring[0];

        // ---- two-loop recursion on the Gram matrix.  With ring positions c (oldest first),
        // rho_c = 1 / s_c'y_c, the first loop is the back substitution
        //   alpha_c = rho_c (s_c'g - sum_{d > c} alpha_d s_c'y_d),
        // gamma = s'y / y'y of the newest pair, and the second loop the forward substitution
        //   beta_c = rho_c (gamma (y_c'g - sum_d alpha_d y_c'y_d) + sum_{d < c} w_d y_c's_d),
        // w_d = alpha_d - beta_d; then -H g = -gamma g + gamma sum_c alpha_c y_c - sum_c w_c s_c.
        // Lane c holds row c; each substitution step is one broadcast.
        const bool act = lane < count;
        const int sl = act ? ring[2 + lane] : 0;
        const vec_t rho = act ? vec_t(1) / Gm[sl * kBasis + KS + sl] : vec_t(0);
        vec_t acc = act ? S.ob[pa_idx(sl, 0)] : vec_t(0);
        vec_t my_alpha = 0, my_w = 0, gam = 1;
        for (int cc = count - 1; cc >= 0; --cc) {
          const vec_t a = __shfl_sync(0xffffffffu, rho * acc, cc);
          if (lane == cc) my_alpha = a;
          const int slc = ring[2 + cc];
          if (lane < cc) acc -= a * Gm[sl * kBasis + KS + slc];
        }
        if (count > 0) {
          const int nw_ = ring[2 + count - 1];
          gam = Gm[nw_ * kBasis + KS + nw_] / Gm[(KS + nw_) * kBasis + KS + nw_];
        }
        vec_t t = act ? S.ob[pa_idx(sl, 1)] : vec_t(0);
        for (int dd = 0; dd < count; ++dd) {
          const vec_t ad = __shfl_sync(0xffffffffu, my_alpha, dd);
          const int sld = ring[2 + dd];
          if (act) t -= ad * Gm[(KS + sl) * kBasis + KS + sld];
        }
        vec_t acc2 = gam * t;
        for (int cc = 0; cc < count; ++cc) {
          const vec_t bcc = __shfl_sync(0xffffffffu, rho * acc2, cc);
          const vec_t w = __shfl_sync(0xffffffffu, my_alpha, cc) - bcc;
          if (lane == cc) my_w = w;
          const int slc = ring[2 + cc];
          if (act && lane > cc) acc2 += w * Gm[slc * kBasis + KS + sl];
        }
        if (act) {
          S.coef[sl] = -my_w;
          S.coef[KS + sl] = gam * my_alpha;
        }
        const unsigned used = __reduce_or_sync(0xffffffffu, act ? (1u << sl) : 0u);
        if (lane == 0) { S.coef[GI] = -gam; S.used = used; }
      }
      rbuf ^= 1;
      __syncthreads();
      const acc_t Ep = fresh ? E : S.eA;
      const vec_t gg = S.ob[PA_GG];
      const sc_t gnorm = sqrt((sc_t)gg);
      gsum += gnorm;
      fresh = false;
      if (!(gnorm > sc_t(0))) {
        if (!isfinite((float)gnorm)) status = 5;
        continue;
      }

      bool accepted = false;
      acc_t Et = 0;
      vec_t disp2 = 0;
      for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
        if (attempt == 1) {
          if (ring[0] == 0) break;
          __syncthreads();
          if (tid == 0) { ring[0] = 0; S.used = 0u; }
          ++resets;
          for (int u = tid; u < kBasis; u += T) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
          __syncthreads();
        }
        // ---- pass B: direction, g'd and the largest per-circle move.  Two positions per thread at a
        // time, so that the secant-slot loads of both are in flight together; g'd takes the positions
        // in the same order as one at a time.
        acc_t gdB = 0;
        vec_t dmB = 0;
        for (int round = 0; round < 2; ++round) {
          const unsigned used = S.used;
          gdB = 0;
          dmB = 0;
          for (int pos = b + tid; pos < e; pos += 2 * T) {
            const int p2 = pos + T;
            const bool h2 = p2 < e;
            const int q2 = h2 ? p2 : pos;
            const VV gi = g[pos], gi2 = g[q2];
            const vec_t cg = S.coef[GI];
            vec_t dx = cg * gi.x, dy = cg * gi.y;
            vec_t dx2 = cg * gi2.x, dy2 = cg * gi2.y;
#pragma unroll
            for (int a = 0; a < kMaxSlots; ++a) {
              if (a < mm && ((used >> a) & 1u)) {
                const VV s_ = Sv[(int64_t)a * n + pos], y_ = Yv[(int64_t)a * n + pos];
                const VV s2 = Sv[(int64_t)a * n + q2], y2 = Yv[(int64_t)a * n + q2];
                const vec_t cs = S.coef[a], cy = S.coef[KS + a];
                dx += cs * s_.x + cy * y_.x;
                dy += cs * s_.y + cy * y_.y;
                dx2 += cs * s2.x + cy * y2.x;
                dy2 += cs * s2.y + cy * y2.y;
              }
            }
            VV dd; dd.x = dx; dd.y = dy;
            dv[pos] = dd;
            gdB += (acc_t)(gi.x * dx + gi.y * dy);
            dmB = max(dmB, dx * dx + dy * dy);
            if (h2) {
              VV d2; d2.x = dx2; d2.y = dy2;
              dv[p2] = d2;
              gdB += (acc_t)(gi2.x * dx2 + gi2.y * dy2);
              dmB = max(dmB, dx2 * dx2 + dy2 * dy2);
            }
          }
          reduce_sm<A, W>(S, rbuf, gdB, dmB);
          if (gdB < acc_t(0) || round == 1) break;
          // not a descent direction: drop the memory, take -g
          if (tid == 0) { ring[0] = 0; S.used = 0u; }
          if (used != 0u) ++resets;
          for (int u = tid; u < kBasis; u += T) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
          __syncthreads();
        }
        const sc_t gd = (sc_t)gdB;
        const sc_t dmax = sqrt((sc_t)dmB);
        if (!(gd < sc_t(0))) break;
        sc_t al = (dmax > step_max) ? step_max / dmax : sc_t(1);
        for (int tr = 0; tr < P.max_trials; ++tr) {
          // ---- pass C: trial coordinates
          for (int pos = b + tid; pos < e; pos += T) {
            PP xo_ = xo[pos];
            VV dd = dv[pos];
            PP v;
            v.x = xo_.x + (pos_t)(al * (sc_t)dd.x);
            v.y = xo_.y + (pos_t)(al * (sc_t)dd.y);
            xw[pos] = v;
          }
          __syncthreads();
          // ---- pass D: trial batch energy and gradient, displacement since the build
          acc_t aD = 0;
          vec_t cD = 0;
          for (int pos = b + tid; pos < e; pos += T) {
            PP xi = xw[pos];
            vec_t gx = 0, gy = 0;
            acc_t ei = 0;
            row_terms<A, PP>(xi, col, rp[pos], re[pos], xw, b, e, pos, gx, gy, ei);
            vec_t fx, fy;
            acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
            gx += fx; gy += fy;
            aD += ei + d0 * d0;
            VV gg_; gg_.x = gx; gg_.y = gy;
            gt[pos] = gg_;
            PP x0 = xb[pos];
            vec_t ex = (vec_t)(xi.x - x0.x), ey = (vec_t)(xi.y - x0.y);
            cD = max(cD, ex * ex + ey * ey);
          }
          reduce_sm<A, W>(S, rbuf, aD, cD);
          ++trials;
          Et = aD;
          if (Et <= Ep + c1 * al * gd) {
            accepted = true;
            disp2 = cD;
            break;
          }
          al *= sc_t(0.5);
        }
        if (!accepted) {
          for (int pos = b + tid; pos < e; pos += T) xw[pos] = xo[pos];
          __syncthreads();
        }
      }
      if (!accepted) { ++stalls; continue; }
      moved = 1;
      Dmax = max(Dmax, (sc_t)sqrt((sc_t)disp2));

      // ---- pass E: the secant pair s = x_new - x_old, y = g_new - g_old goes to the stage slot;
      // its dots and its curvature test come with this batch's next step
      {
        const int stg = ring[1];
        for (int pos = b + tid; pos < e; pos += T) {
          PP xn = xw[pos], x0 = xo[pos];
          VV s_; s_.x = (vec_t)(xn.x - x0.x); s_.y = (vec_t)(xn.y - x0.y);
          VV gn = gt[pos], go = g[pos];
          VV y_; y_.x = gn.x - go.x; y_.y = gn.y - go.y;
          Sv[(int64_t)stg * n + pos] = s_;
          Yv[(int64_t)stg * n + pos] = y_;
        }
        // every thread raises the flag: with one batch the next read comes without a barrier in
        // between, and each thread then reads its own store (thread 0 clears the flag only after
        // the next step's reduction barriers)
        ring[2 + kMaxSlots] = 1;
        if (k == 1) { fresh = true; E = Et; }
      }
    }
    if (status != 3) break;
    // ---- ANM after the sweep (Algorithm ANM)
    if (P.anm) {
      ++cnt;
      if (cnt >= len) {
        if (!anm_rebuild()) { status = 4; break; }
      }
    }
    // the FP32 phase needs the total energy only for its stagnation check (its e_tol is out of
    // binary32's reach); the FP64 phases test E <= e_tol after every sweep
    const bool check_now = A::kId != 1 || P.stall_window <= 0 || iters % P.stall_window == 0;
    if (check_now && !(k == 1 && fresh)) { E = full_energy(); e_at = iters; }
    if (k == 1 && fresh) e_at = iters;
    if (!isfinite(E)) { status = 5; break; }
    if (E <= (acc_t)P.e_tol) { status = 0; break; }
    if (gsum <= gsum_tol) { status = 1; break; }
    if (!moved) { status = 2; break; }
    // FP32 phase: binary32 has reached its resolution when E stops falling, hand over; polish: a
    // run whose E stops falling above zero sits at a jammed local minimum
    if (A::kId != 0 && P.stall_window > 0 && iters % P.stall_window == 0) {
      if (E > Ewin * (acc_t)(1.0 - P.stall_rel)) { status = 2; break; }
      Ewin = E;
    }
    if (P.budget_ns > 0) {
      if (tid == 0) S.flag = globaltimer_ns() - *P.t0 > P.budget_ns;
      __syncthreads();
      int late = S.flag;
      __syncthreads();
      if (late) { status = 6; break; }
    }
  }

  if (status < 4 && e_at != iters) E = full_energy();  // the final energy of the run
  // ---- parity hook: the lists in force now, in the caller's numbering, and their build's layout
  if (P.dump_cnt != nullptr) {
    const int64_t stride = P.dump_stride;
    for (int pos = tid; pos < n; pos += T) {
      const int i = perm[pos];
      const int b0 = lists_ok ? rp[pos] : 0, len_ = lists_ok ? re[pos] - b0 : 0;
      const bool ok = lists_ok && len_ <= P.dump_stride;
      P.dump_cnt[D.off + i] = ok ? len_ : -1;
      if (ok)
        for (int t = 0; t < len_; ++t) P.dump_col[(D.off + i) * stride + t] = perm[col[b0 + t]];
      const PP v = xb[pos];
      P.dump_xb[D.off + i] = make_double2((double)v.x, (double)v.y);
    }
  }
  // ---- 4. merge: scatter back to the caller's order
  for (int pos = tid; pos < n; pos += T) {
    int i = perm[pos];
    PP v = xw[pos];
    if (A::kId == 1) {
      P.x32[D.off + i] = make_float2((float)v.x, (float)v.y);
    } else {
      P.x64[D.off + i] = make_double2((double)v.x, (double)v.y);
      if (A::kId == 2) P.x32[D.off + i] = make_float2((float)v.x, (float)v.y);
    }
  }
  if (tid == 0) {
    if (A::kId == 1) {
      O->iters32 = iters; O->status32 = status; O->E32 = (double)E; O->trials32 = trials;
      O->iters = iters; O->status = status; O->E = (double)E; O->polished = 0;
      O->builds = builds; O->changes = changes; O->trials = trials; O->resets = resets; O->stalls = stalls;
    } else if (A::kId == 2) {
      O->iters = O->iters32 + iters; O->status = status; O->E = (double)E; O->polished = 1;
      O->builds += builds; O->changes += changes; O->trials += trials; O->resets += resets; O->stalls += stalls;
    } else {
      O->iters = iters; O->status = status; O->E = (double)E; O->polished = 0;
      O->builds = builds; O->changes = changes; O->trials = trials; O->resets = resets; O->stalls = stalls;
      O->iters32 = iters; O->trials32 = trials;
    }
  }
  __syncthreads();
}

// MAXT: threads per block, at most; MINB: resident blocks per SM the register budget is sized for
template <class A, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
descend_kernel(DescendParams P) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Smem<A, MAXT / 32> S;
  const int num = P.num_dev ? *P.num_dev : P.num;
  for (;;) {
    if (threadIdx.x == 0) S.q = atomicAdd(P.queue, 1);
    __syncthreads();
    const int qi = S.q;
    __syncthreads();
    if (qi >= num) break;
    descend_instance<A, MAXT / 32>(P, S, dsm, P.order[qi]);
  }
}

// The FP32 descent and the FP64 polish of each instance back to back in the same block: no
// grid-wide gap between the phases, so long polishes overlap other instances' FP32 descents.
// P32 / P64: the two phases' parameters (the dynamic shared memory is the larger share of the two).
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
descend_fused_kernel(DescendParams P32, DescendParams P64) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Smem<Arith32, MAXT / 32> S32;
  __shared__ Smem<ArithMix, MAXT / 32> S64;
  const int num = P32.num_dev ? *P32.num_dev : P32.num;
  for (;;) {
    if (threadIdx.x == 0) S32.q = atomicAdd(P32.queue, 1);
    __syncthreads();
    const int qi = S32.q;
    __syncthreads();
    if (qi >= num) break;
    const int q = P32.order[qi];
    descend_instance<Arith32, MAXT / 32>(P32, S32, dsm, q);
    descend_instance<ArithMix, MAXT / 32>(P64, S64, dsm, q);
  }
}

// One compiled instance of the descent kernel: its launch bound and the static shared memory of
// its block state.
template <class A, int MAXT, int MINB> DescendVariant descend_variant() {
  return DescendVariant{(const void *)descend_kernel<A, MAXT, MINB>, MAXT, MINB, sizeof(Smem<A, MAXT / 32>)};
}
template <int MAXT, int MINB> DescendVariant descend_fused_variant() {
  return DescendVariant{(const void *)descend_fused_kernel<MAXT, MINB>, MAXT, MINB,
                        sizeof(Smem<Arith32, MAXT / 32>) + sizeof(Smem<ArithMix, MAXT / 32>)};
}

}  // namespace
}  // namespace pecc
