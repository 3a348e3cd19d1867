// pecc_grid.cu -- descent of ONE large instance by the whole GPU: Algorithm GBO (Sec. 4.1) with
// ANM (Sec. 4.3), the steps of descend_kernel with every block-wide step made grid-wide.
//
// One cooperative launch (every block resident) runs the whole descent.  Blocks meet at a grid
// barrier built here (an arrival counter and a generation word in global memory); every wait is
// bounded by %globaltimer and raises an error flag instead of spinning on.  Reductions: each block
// reduces its part, block 0 adds the parts, every block reads the totals.  All control decisions,
// the secant-pair ring, the Gram matrices and the two-loop recursion are computed redundantly and
// identically by every block from those totals, so they need no further synchronisation.
//   partition   pseudo-angle (annulus: radius, fence: x) keys; buckets by key value (monotone),
//               counting sort into buckets, per-bucket sort by (key, index): the exact stable order
//   lists       cell keys, counting sort by cell, per-cell index order, coordinates in cell order,
//               count pass, grid scan, fill pass with a digest of the pair set (for ANM)
//   batch step  pass A (E_p, g, dots incl. the pending pair), push + two-loop, pass B (direction),
//               trials (C: coordinates, D: energy and gradient at the trial), pass E (s, y)
#include "pecc_internal.h"

namespace pecc {
namespace {

constexpr int KS = kMaxSlots;
constexpr int GI = 2 * kMaxSlots;
constexpr int OP = 1 + 2 * kMaxSlots;
constexpr int NV1 = OP + 4 * kMaxSlots + 3;  // values of the first reduction of a batch step
constexpr int kPart = 72;                    // stride of a block's partials (>= NV1 + 2)
constexpr int kRing = kMaxSlots + 4;         // count, stage, ring[kMaxSlots], pending, used
constexpr long long kBarrierTimeoutNs = 2000000000ll;

__device__ __forceinline__ unsigned ldv(const unsigned *p) { return *(volatile const unsigned *)p; }
__device__ __forceinline__ int ldv(const int *p) { return *(volatile const int *)p; }

// Grid barrier for `expected` arriving blocks; false (for the whole block) once any block's wait
// has run past timeout_ns (measured on %globaltimer) and raised the shared error flag.
__device__ bool grid_sync_n(GridCtl *c, unsigned expected, long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ldv(&c->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&c->count, 1u) + 1u;
    int good = 1;
    if (arrived == expected) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      const long long t0 = globaltimer_ns();
      while (ldv(&c->gen) == g) {
        if (ldv(&c->err)) { good = 0; break; }
        if (globaltimer_ns() - t0 > timeout_ns) { atomicExch(&c->err, 1); good = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good && !ldv(&c->err);
  }
  __syncthreads();
  return ok;
}

__device__ __forceinline__ bool grid_sync(GridCtl *c) { return grid_sync_n(c, gridDim.x, kBarrierTimeoutNs); }

template <class A> struct GSmem {
  using vec_t = typename A::vec_t;
  double wb[16 * kPart];       // per-warp partials
  double tot[kPart];           // reduction totals
  vec_t gram[kBasis * kBasis]; // Gram matrix of the current batch (identical in every block)
  vec_t coef[kBasis];
  int ring[kMaxK][kRing];
  int32_t sh[40];
  long long iv[2];
  int flag;
  int rbuf;  // partial buffer of the next grid_reduce (same in every block)
};

// Grid-wide reduction of NV values (kind 0: sum, 1: max) with one grid barrier: every block writes
// its partials to buffer S.rbuf of G.part, and after the barrier every block combines all blocks'
// partials itself (warp q takes value q, its lanes stride over the blocks, then a fixed butterfly),
// so every block holds bit-identical totals in S.tot[].  Consecutive reductions alternate the two
// buffers: a block writes a buffer again only after the next reduction's barrier, which every
// block passes after its reads of this one.
template <class A, int NV, typename T>
__device__ bool grid_reduce(GSmem<A> &S, const GridBufs &G, GridCtl *c, T (&v)[NV], const int (&kind)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int buf = S.rbuf;
  double *part = G.part + (size_t)buf * gridDim.x * kPart;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    T s = kind[q] ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0) S.wb[w * kPart + q] = (double)s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NV; q += blockDim.x) {
    double s = S.wb[q];
    for (int u = 1; u < nw; ++u) s = kind[q] ? fmax(s, S.wb[u * kPart + q]) : s + S.wb[u * kPart + q];
    part[(size_t)blockIdx.x * kPart + q] = s;
  }
  if (!grid_sync(c)) return false;
  if (NV <= 8) {
    for (int q = w; q < NV; q += nw) {
      double s = kind[q] ? -INFINITY : 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) {
        const double x = __ldcg(part + (size_t)b * kPart + q);  // L2: another block wrote it
        s = kind[q] ? fmax(s, x) : s + x;
      }
      s = kind[q] ? warp_max(s) : warp_sum(s);
      if (lane == 0) S.tot[q] = s;
    }
  } else {
    // many values: block q combines value q over all blocks and publishes it, then a second
    // barrier, and every block reads the NV totals (instead of every block reading NV x grid
    // partials)
    double *res = G.res + (size_t)buf * kPart;
    for (int q = blockIdx.x; q < NV; q += gridDim.x) {
      double s = kind[q] ? -INFINITY : 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double x = __ldcg(part + (size_t)b * kPart + q);
        s = kind[q] ? fmax(s, x) : s + x;
      }
      s = kind[q] ? warp_max(s) : warp_sum(s);
      if (lane == 0) S.wb[w] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = S.wb[0];
        for (int u = 1; u < nw; ++u) t = kind[q] ? fmax(t, S.wb[u]) : t + S.wb[u];
        res[q] = t;
      }
      __syncthreads();
    }
    if (!grid_sync(c)) return false;
    for (int q = threadIdx.x; q < NV; q += blockDim.x) S.tot[q] = __ldcg(res + q);
  }
  __syncthreads();
  if (threadIdx.x == 0) S.rbuf = buf ^ 1;
  __syncthreads();
  return true;
}

// Inclusive prefix sum of a[0..len) in place across the grid (each block one contiguous chunk);
// the total goes to S.iv[1].  False on a barrier failure.
template <class A>
__device__ bool grid_scan(GSmem<A> &S, const GridBufs &G, GridCtl *c, int32_t *a, int len) {
  const int nb = gridDim.x, b = blockIdx.x;
  const int chunk = (len + nb - 1) / nb;
  const int lo = min(len, b * chunk), hi = min(len, lo + chunk);
  block_scan_inplace(a + lo, hi - lo, S.sh);
  if (threadIdx.x == 0) G.ipart[b] = (hi > lo) ? a[hi - 1] : 0;
  if (!grid_sync(c)) return false;
  if (threadIdx.x == 0) {
    long long off = 0, tot = 0;
    for (int u = 0; u < nb; ++u) {
      const int v = *(volatile const int *)&G.ipart[u];
      if (u < b) off += v;
      tot += v;
    }
    S.iv[0] = off;
    S.iv[1] = tot;
  }
  __syncthreads();
  const int off = (int)S.iv[0];
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) a[i] += off;
  return grid_sync(c);
}

template <class A>
__global__ void __launch_bounds__(256, 1) descend_grid_kernel(DescendParams P, int q, GridBufs G, GridCtl *ctl) {
  using pos_t = typename A::pos_t;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  using sc_t = acc_t;
  using PP = v2<pos_t>;
  using VV = v2<vec_t>;
  __shared__ GSmem<A> S;
  const int tid = threadIdx.x;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  const InstDesc D = P.desc[q];
  InstOut *O = P.out + q;
  const int n = D.n;
  const int mm = P.m + 1;
  const acc_t R = (acc_t)D.R;
  const acc_t Rm1sq = (acc_t)((D.R >= 1.0) ? (D.R - 1.0) * (D.R - 1.0) : -1.0);
  const sc_t c1 = (sc_t)P.c1, step_max = (sc_t)P.step_max, two_skin = (sc_t)(2.0 * P.rebuild_disp);
  const sc_t gsum_tol = (sc_t)P.gsum_tol, curv_eps = (sc_t)P.curv_eps;

  if (tid == 0) S.rbuf = 0;
  __syncthreads();
  if (A::kId == 2) {  // the polish runs only on instances the FP32 descent left near zero energy
    if (!(O->E32 <= P.polish_gate) || O->status32 >= 4) {
      for (int i = gid; i < n; i += gstride) {
        float2 v = P.x32[D.off + i];
        P.x64[D.off + i] = make_double2((double)v.x, (double)v.y);
      }
      if (gid == 0) { O->iters = O->iters32; O->status = O->status32; O->E = O->E32; O->polished = 0; }
      return;
    }
  }
  const int k = (P.k_override > 0) ? min(P.k_override, D.k) : D.k;
  PP *xw = (PP *)((double2 *)P.xw + D.off), *xb = (PP *)((double2 *)P.xb + D.off), *xo = (PP *)((double2 *)P.xo + D.off);
  VV *g = (VV *)((double2 *)P.g + D.off), *gt = (VV *)((double2 *)P.gt + D.off), *dv = (VV *)((double2 *)P.d + D.off);
  VV *Sv = (VV *)P.S + (int64_t)mm * D.off, *Yv = (VV *)P.Y + (int64_t)mm * D.off;
  int32_t *perm = P.perm + D.off;
  uint64_t *skey = P.skey + D.off;
  int32_t *rp = P.rp + D.rp_off;
  int32_t *col = P.col + D.col_off;
  const int cap = 2 * D.cap;
  uint32_t *ckey = P.ckey + D.off;
  int32_t *corder = P.corder + D.off;
  int32_t *cells = P.cells + D.cell_off;
  const CellGrid Gc = (A::kId == 1) ? CellGrid{D.R, D.inv_cs, (float)D.R, D.inv_f, D.ncx_f, true}
                                    : CellGrid{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
  const pos_t lc2 = (pos_t)(P.l_cut * P.l_cut);
  int status = 3;
  bool ok = true;

  // ---- 1. partition: keys, their range, buckets by value, per-bucket (key, index) order
  const int nbk = max(1, n / 4);
  {
    double kmax = -1e300, kmin_neg = -1e300;
    for (int i = gid; i < n; i += gstride) {
      double x, y;
      if (A::kId == 0) { double2 v = P.x64[D.off + i]; x = v.x; y = v.y; }
      else { float2 v = P.x32[D.off + i]; x = v.x; y = v.y; }
      const double key = P.partition == 3 ? random_part_key(P.part_seed, i, q) : part_key(x, y, P.partition);
      skey[i] = sortable(key);
      kmax = fmax(kmax, key);
      kmin_neg = fmax(kmin_neg, -key);
    }
    for (int c = gid; c <= 2 * nbk; c += gstride) G.bucket[c] = 0;
    double v[2] = {kmax, kmin_neg};
    const int kind[2] = {1, 1};
    ok = grid_reduce<A, 2, double>(S, G, ctl, v, kind);
  }
  const double kmin = -S.tot[1], krange = S.tot[0] - kmin;
  const bool finite_keys = isfinite(kmin) && isfinite(krange);
  auto bucket_of = [&](uint64_t sk) -> int {
    // invert the sortable map to the key, then a monotone bucket index
    uint64_t b = (sk & 0x8000000000000000ull) ? (sk & 0x7fffffffffffffffull) : ~sk;
    double key = __longlong_as_double((long long)b);
    if (!(krange > 0.0) || !finite_keys) return 0;
    double f = (key - kmin) / krange * (double)nbk;
    int bi = (f >= 0.0) ? (int)f : 0;
    return bi >= nbk ? nbk - 1 : bi;
  };
  if (ok) {
    for (int i = gid; i < n; i += gstride) atomicAdd(&G.bucket[bucket_of(skey[i]) + 1], 1);
    ok = grid_sync(ctl) && grid_scan(S, G, ctl, G.bucket + 1, nbk);
  }
  if (ok) {
    int32_t *bfill = G.bucket + nbk + 1;
    for (int c = gid; c < nbk; c += gstride) bfill[c] = G.bucket[c];
    ok = grid_sync(ctl);
    if (ok) {
      for (int i = gid; i < n; i += gstride) perm[atomicAdd(&bfill[bucket_of(skey[i])], 1)] = i;
      ok = grid_sync(ctl);
    }
  }
  if (ok) {
    for (int c = gid; c < nbk; c += gstride) {  // insertion sort of a bucket by (key, index)
      const int lo = G.bucket[c], hi = G.bucket[c + 1];
      for (int a = lo + 1; a < hi; ++a) {
        const int v = perm[a];
        const uint64_t kv = skey[v];
        int b = a - 1;
        while (b >= lo) {
          const int u = perm[b];
          const uint64_t ku = skey[u];
          if (ku < kv || (ku == kv && u < v)) break;
          perm[b + 1] = u;
          --b;
        }
        perm[b + 1] = v;
      }
    }
    ok = grid_sync(ctl);
  }
  // ---- 2. renumber in partition order
  int bad = 0;
  if (ok) {
    for (int p = gid; p < n; p += gstride) {
      const int i = perm[p];
      PP v;
      if (A::kId == 0) { double2 u = P.x64[D.off + i]; v.x = (pos_t)u.x; v.y = (pos_t)u.y; }
      else { float2 u = P.x32[D.off + i]; v.x = (pos_t)u.x; v.y = (pos_t)u.y; }
      bad |= !(isfinite((float)v.x) && isfinite((float)v.y));
      xw[p] = v;
      xb[p] = v;
    }
    double vb[1] = {(double)bad};
    const int kind[1] = {1};
    ok = grid_reduce<A, 1, double>(S, G, ctl, vb, kind);
    bad = ok && S.tot[0] > 0.0;
  }

  int iters = 0, builds = 0, changes = 0, trials = 0, resets = 0, stalls = 0;
  int cnt = 0, len = 1;
  unsigned long long hcur = 0ull;
  sc_t Dmax = 0;
  acc_t E = 0;

  // ---- neighbor lists over the grid; false on overflow or a barrier failure (status set)
  auto build = [&]() -> bool {
    const int ncell = Gc.nc * Gc.nc;
    int32_t *cstart = cells, *cfill = cells + ncell + 1;
    for (int c = gid; c <= ncell; c += gstride) cstart[c] = 0;
    if (gid == 0) { *G.hash = 0ull; rp[0] = 0; }
    if (!grid_sync(ctl)) return false;
    for (int i = gid; i < n; i += gstride) {
      const uint32_t key = grid_key<pos_t>(xw[i], Gc);
      ckey[i] = key;
      atomicAdd(&cstart[key + 1], 1);
    }
    if (!grid_sync(ctl) || !grid_scan(S, G, ctl, cstart + 1, ncell)) return false;
    for (int c = gid; c < ncell; c += gstride) cfill[c] = cstart[c];
    if (!grid_sync(ctl)) return false;
    for (int i = gid; i < n; i += gstride) corder[atomicAdd(&cfill[ckey[i]], 1)] = i;
    if (!grid_sync(ctl)) return false;
    for (int c = gid; c < ncell; c += gstride) {
      const int lo = cstart[c], hi = cstart[c + 1];
      for (int a = lo + 1; a < hi; ++a) {
        const int v = corder[a];
        int b = a - 1;
        while (b >= lo && corder[b] > v) { corder[b + 1] = corder[b]; --b; }
        corder[b + 1] = v;
      }
    }
    if (!grid_sync(ctl)) return false;
    for (int p = gid; p < n; p += gstride) xo[p] = xw[corder[p]];  // coordinates in cell order
    if (!grid_sync(ctl)) return false;
    const int nc = Gc.nc;
    for (int q0 = gid; q0 < n; q0 += gstride) {
      const int i = corder[q0];
      const PP xi = xo[q0];
      const uint32_t key = ckey[i];
      const int cx = (int)(key % (uint32_t)nc), cy = (int)(key / (uint32_t)nc);
      const int bx0 = max(cx - 1, 0), bx1 = min(cx + 1, nc - 1);
      int cntn = 0;
      for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by) {
        const int lo = cstart[by * nc + bx0], hi = cstart[by * nc + bx1 + 1];
        for (int qq = lo; qq < hi; ++qq) cntn += nbr_pred(xi, xo[qq], lc2) && qq != q0;
      }
      rp[i + 1] = cntn;
    }
    if (!grid_sync(ctl) || !grid_scan(S, G, ctl, rp + 1, n)) return false;
    const long long total = S.iv[1];
    if (total > cap) { status = 4; return false; }
    unsigned long long h = 0ull;
    for (int q0 = gid; q0 < n; q0 += gstride) {
      const int i = corder[q0];
      const PP xi = xo[q0];
      const uint32_t key = ckey[i];
      const int cx = (int)(key % (uint32_t)nc), cy = (int)(key / (uint32_t)nc);
      const int bx0 = max(cx - 1, 0), bx1 = min(cx + 1, nc - 1);
      int w = rp[i];
      for (int by = max(cy - 1, 0); by <= min(cy + 1, nc - 1); ++by) {
        const int lo = cstart[by * nc + bx0], hi = cstart[by * nc + bx1 + 1];
        for (int qq = lo; qq < hi; ++qq) {
          if (nbr_pred(xi, xo[qq], lc2) && qq != q0) {
            const int j = corder[qq];
            col[w++] = j;
            h += mix32((uint32_t)i * 0x9E3779B1u ^ (uint32_t)j);
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((tid & 31) == 0) atomicAdd(G.hash, h);
    if (!grid_sync(ctl)) return false;
    return true;
  };
  auto anm_rebuild = [&]() -> bool {
    if (!build()) return false;
    ++builds;
    const unsigned long long h = *(volatile unsigned long long *)G.hash;
    if (h != hcur) { hcur = h; len = 1; ++changes; }
    else if (len < (1 << 30)) len *= 2;
    cnt = 0;
    for (int p = gid; p < n; p += gstride) xb[p] = xw[p];
    Dmax = 0;
    return grid_sync(ctl);
  };
  auto full_energy = [&](bool &good) -> acc_t {
    double e = 0.0;
    for (int p = gid; p < n; p += gstride) {
      const PP xi = xw[p];
      acc_t ei = 0;
      for (int t = rp[p]; t < rp[p + 1]; ++t) {
        const int j = col[t];
        if (j >= p) continue;
        vec_t fx, fy;
        const acc_t d = A::pair(xi, xw[j], fx, fy);
        ei += d * d;
      }
      vec_t fx, fy;
      const acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
      e += (double)(ei + d0 * d0);
    }
    double v[1] = {e};
    const int kind[1] = {0};
    good = grid_reduce<A, 1, double>(S, G, ctl, v, kind);
    return (acc_t)S.tot[0];
  };

  if (!ok) status = 6;
  else if (bad) status = 5;
  else if (!build()) { if (status == 3) status = 6; }
  else {
    builds = 1;
    hcur = *(volatile unsigned long long *)G.hash;
    bool good = true;
    E = full_energy(good);
    if (!good) status = 6;
    else if (!isfinite(E)) status = 5;
    else if (E <= (acc_t)P.e_tol) status = 0;
  }
  for (int u = tid; u < k * kRing; u += blockDim.x) S.ring[u / kRing][u % kRing] = 0;
  // every block keeps identical Gram matrices (built from identical totals) in its own slice
  vec_t *gram_mine = (vec_t *)G.gram + (size_t)blockIdx.x * G.kmax * kBasis * kBasis;
  for (int u = tid; u < k * kBasis * kBasis; u += blockDim.x) gram_mine[u] = vec_t(0);
  __syncthreads();

  const int q_ = n / k, r_ = n % k;
  bool fresh = false;
  int e_at = 0;
  acc_t Ewin = E;

  while (status == 3 && iters < P.max_iter) {
    ++iters;
    sc_t gsum = 0;
    int moved = 0;
    for (int p = 0; p < k && status == 3; ++p) {
      const int b = p * q_ + min(p, r_), e = b + q_ + (p < r_ ? 1 : 0);
      if (sc_t(2) * Dmax + step_max > two_skin) {
        if (!anm_rebuild()) { if (status == 3) status = 6; break; }
        fresh = false;
      }
      int *ring = S.ring[p];
      vec_t *Gm = gram_mine + (size_t)p * kBasis * kBasis;
      const int count0 = ring[0], st = ring[1], pending = ring[2 + KS];
      // ---- pass A
      double vA[NV1 + 1];  // the dots, and the batch energy last
      int kindA[NV1 + 1];
#pragma unroll
      for (int u = 0; u <= NV1; ++u) { vA[u] = 0.0; kindA[u] = 0; }
      if (fresh) { VV *t_ = g; g = gt; gt = t_; }
      for (int pos = b + gid; pos < e; pos += gstride) {
        const PP xi = xw[pos];
        xo[pos] = xi;
        VV gi;
        if (!fresh) {
          vec_t gx = 0, gy = 0;
          acc_t ei = 0;
          for (int t = rp[pos]; t < rp[pos + 1]; ++t) {
            const int j = col[t];
            vec_t fx, fy;
            const acc_t d = A::pair(xi, xw[j], fx, fy);
            gx += fx; gy += fy;
            if (j < b || j >= e || j < pos) ei += d * d;
          }
          vec_t fx, fy;
          const acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
          gx += fx; gy += fy;
          vA[NV1] += (double)(ei + d0 * d0);
          gi.x = gx; gi.y = gy;
          g[pos] = gi;
        } else {
          gi = g[pos];
        }
        vA[0] += (double)(gi.x * gi.x + gi.y * gi.y);
        VV sp, yp;
        if (pending) { sp = Sv[(int64_t)st * n + pos]; yp = Yv[(int64_t)st * n + pos]; }
#pragma unroll
        for (int a = 0; a < kMaxSlots; ++a) {
          if (a < mm) {
            const VV s_ = Sv[(int64_t)a * n + pos], y_ = Yv[(int64_t)a * n + pos];
            vA[1 + a] += (double)(gi.x * s_.x + gi.y * s_.y);
            vA[1 + KS + a] += (double)(gi.x * y_.x + gi.y * y_.y);
            if (pending) {
              vA[OP + a] += (double)(sp.x * s_.x + sp.y * s_.y);
              vA[OP + KS + a] += (double)(sp.x * y_.x + sp.y * y_.y);
              vA[OP + 2 * KS + a] += (double)(yp.x * s_.x + yp.y * s_.y);
              vA[OP + 3 * KS + a] += (double)(yp.x * y_.x + yp.y * y_.y);
            }
          }
        }
        if (pending) {
          vA[OP + 4 * KS + 0] += (double)(sp.x * sp.x + sp.y * sp.y);
          vA[OP + 4 * KS + 1] += (double)(sp.x * yp.x + sp.y * yp.y);
          vA[OP + 4 * KS + 2] += (double)(yp.x * yp.x + yp.y * yp.y);
        }
      }
      if (!grid_reduce<A, NV1 + 1, double>(S, G, ctl, vA, kindA)) { status = 6; break; }
      const acc_t Ep = fresh ? E : (acc_t)S.tot[NV1];
      const vec_t gg = (vec_t)S.tot[0];
      const sc_t gnorm = sqrt((sc_t)gg);
      gsum += gnorm;
      fresh = false;
      if (pending) {  // curvature test and push (identical in every block)
        const vec_t ss = (vec_t)S.tot[OP + 4 * KS], sy = (vec_t)S.tot[OP + 4 * KS + 1],
                    yy = (vec_t)S.tot[OP + 4 * KS + 2];
        const bool push = (sc_t)sy > curv_eps * sqrt((sc_t)ss) * sqrt((sc_t)yy) && P.m > 0;
        if (push) {
          if (tid < count0) {
            const int sl = ring[2 + tid];
            Gm[st * kBasis + sl] = Gm[sl * kBasis + st] = (vec_t)S.tot[OP + sl];
            Gm[st * kBasis + KS + sl] = Gm[(KS + sl) * kBasis + st] = (vec_t)S.tot[OP + KS + sl];
            Gm[(KS + st) * kBasis + sl] = Gm[sl * kBasis + KS + st] = (vec_t)S.tot[OP + 2 * KS + sl];
            Gm[(KS + st) * kBasis + KS + sl] = Gm[(KS + sl) * kBasis + KS + st] = (vec_t)S.tot[OP + 3 * KS + sl];
          }
          if (tid == 0) {
            Gm[st * kBasis + st] = ss;
            Gm[st * kBasis + KS + st] = Gm[(KS + st) * kBasis + st] = sy;
            Gm[(KS + st) * kBasis + KS + st] = yy;
          }
        }
        __syncthreads();
        if (tid == 0) {
          if (push) {
            const int c = ring[0];
            if (c < P.m) {
              ring[2 + c] = st;
              ring[0] = c + 1;
              int fr = 0;
              for (; fr < mm; ++fr) {
                bool used = false;
                for (int u = 0; u <= c; ++u) used |= (ring[2 + u] == fr);
                if (!used) break;
              }
              ring[1] = fr;
            } else {
              const int ev = ring[2];
              for (int u = 0; u + 1 < c; ++u) ring[2 + u] = ring[3 + u];
              ring[2 + c - 1] = st;
              ring[1] = ev;
            }
          }
          ring[2 + KS] = 0;
        }
        __syncthreads();
      }
      const int count = ring[0];
      if (!(gnorm > sc_t(0))) {
        if (!isfinite((float)gnorm)) status = 5;
        continue;
      }
      // ---- two-loop (warp 0 of every block, identical results)
      if (tid < 32) {
        const int lane = tid;
        const bool act = lane < count;
        const int sl = act ? ring[2 + lane] : 0;
        const vec_t rho = act ? vec_t(1) / Gm[sl * kBasis + KS + sl] : vec_t(0);
        vec_t acc = act ? (vec_t)S.tot[1 + sl] : vec_t(0);
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
        vec_t t = act ? (vec_t)S.tot[1 + KS + sl] : vec_t(0);
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
        for (int u = lane; u < kBasis; u += 32) S.coef[u] = vec_t(0);
        __syncwarp();
        if (act) { S.coef[sl] = -my_w; S.coef[KS + sl] = gam * my_alpha; }
        if (lane == 0) S.coef[GI] = -gam;
      }
      __syncthreads();

      bool accepted = false;
      acc_t Et = 0;
      double disp2 = 0.0;
      for (int attempt = 0; attempt < 2 && !accepted && status == 3; ++attempt) {
        if (attempt == 1) {
          if (ring[0] == 0) break;
          __syncthreads();
          if (tid == 0) ring[0] = 0;
          ++resets;
          for (int u = tid; u < kBasis; u += blockDim.x) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
          __syncthreads();
        }
        for (int round = 0; round < 2; ++round) {
          const int cnt_now = ring[0];
          double vB[2] = {0.0, 0.0};
          const int kindB[2] = {0, 1};
          for (int pos = b + gid; pos < e; pos += gstride) {
            const VV gi = g[pos];
            const vec_t cg = S.coef[GI];
            vec_t dx = cg * gi.x, dy = cg * gi.y;
            for (int c = 0; c < cnt_now; ++c) {
              const int sl = ring[2 + c];
              const VV s_ = Sv[(int64_t)sl * n + pos], y_ = Yv[(int64_t)sl * n + pos];
              const vec_t cs = S.coef[sl], cy = S.coef[KS + sl];
              dx += cs * s_.x + cy * y_.x;
              dy += cs * s_.y + cy * y_.y;
            }
            VV dd; dd.x = dx; dd.y = dy;
            dv[pos] = dd;
            vB[0] += (double)(gi.x * dx + gi.y * dy);
            vB[1] = fmax(vB[1], (double)(dx * dx + dy * dy));
          }
          if (!grid_reduce<A, 2, double>(S, G, ctl, vB, kindB)) { status = 6; break; }
          if (S.tot[0] < 0.0 || round == 1) break;
          __syncthreads();
          if (tid == 0) ring[0] = 0;
          if (cnt_now > 0) ++resets;
          for (int u = tid; u < kBasis; u += blockDim.x) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
          __syncthreads();
        }
        if (status != 3) break;
        const sc_t gd = (sc_t)S.tot[0];
        const sc_t dmax = sqrt((sc_t)S.tot[1]);
        if (!(gd < sc_t(0))) break;
        sc_t al = (dmax > step_max) ? step_max / dmax : sc_t(1);
        for (int tr = 0; tr < P.max_trials; ++tr) {
          for (int pos = b + gid; pos < e; pos += gstride) {
            const PP xo_ = xo[pos];
            const VV dd = dv[pos];
            PP v;
            v.x = xo_.x + (pos_t)(al * (sc_t)dd.x);
            v.y = xo_.y + (pos_t)(al * (sc_t)dd.y);
            xw[pos] = v;
          }
          if (!grid_sync(ctl)) { status = 6; break; }
          double vD[2] = {0.0, 0.0};
          const int kindD[2] = {0, 1};
          for (int pos = b + gid; pos < e; pos += gstride) {
            const PP xi = xw[pos];
            vec_t gx = 0, gy = 0;
            acc_t ei = 0;
            for (int t = rp[pos]; t < rp[pos + 1]; ++t) {
              const int j = col[t];
              vec_t fx, fy;
              const acc_t d = A::pair(xi, xw[j], fx, fy);
              gx += fx; gy += fy;
              if (j < b || j >= e || j < pos) ei += d * d;
            }
            vec_t fx, fy;
            const acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
            gx += fx; gy += fy;
            vD[0] += (double)(ei + d0 * d0);
            VV gg_; gg_.x = gx; gg_.y = gy;
            gt[pos] = gg_;
            const PP x0 = xb[pos];
            const double ex = (double)(xi.x - x0.x), ey = (double)(xi.y - x0.y);
            vD[1] = fmax(vD[1], ex * ex + ey * ey);
          }
          if (!grid_reduce<A, 2, double>(S, G, ctl, vD, kindD)) { status = 6; break; }
          ++trials;
          Et = (acc_t)S.tot[0];
          if (Et <= Ep + c1 * al * gd) { accepted = true; disp2 = S.tot[1]; break; }
          al *= sc_t(0.5);
        }
        if (status != 3) break;
        if (!accepted) {
          for (int pos = b + gid; pos < e; pos += gstride) xw[pos] = xo[pos];
          if (!grid_sync(ctl)) { status = 6; break; }
        }
      }
      if (status != 3) break;
      if (!accepted) { ++stalls; continue; }
      moved = 1;
      Dmax = max(Dmax, (sc_t)sqrt(disp2));
      // ---- pass E: the new pair to the stage slot (its dots come with this batch's next step)
      {
        const int stg = ring[1];
        for (int pos = b + gid; pos < e; pos += gstride) {
          const PP xn = xw[pos], x0 = xo[pos];
          VV s_; s_.x = (vec_t)(xn.x - x0.x); s_.y = (vec_t)(xn.y - x0.y);
          const VV gn = gt[pos], go = g[pos];
          VV y_; y_.x = gn.x - go.x; y_.y = gn.y - go.y;
          Sv[(int64_t)stg * n + pos] = s_;
          Yv[(int64_t)stg * n + pos] = y_;
        }
        __syncthreads();
        if (tid == 0) ring[2 + KS] = 1;
        __syncthreads();
        if (k == 1) { fresh = true; E = Et; }
      }
    }
    if (status != 3) break;
    if (P.anm) {
      ++cnt;
      if (cnt >= len) {
        if (!anm_rebuild()) { if (status == 3) status = 6; break; }
      }
    }
    const bool check_now = A::kId != 1 || P.stall_window <= 0 || iters % P.stall_window == 0;
    if (check_now && !(k == 1 && fresh)) {
      bool good = true;
      E = full_energy(good);
      if (!good) { status = 6; break; }
      e_at = iters;
    }
    if (k == 1 && fresh) e_at = iters;
    if (!isfinite(E)) { status = 5; break; }
    if (E <= (acc_t)P.e_tol) { status = 0; break; }
    if (gsum <= gsum_tol) { status = 1; break; }
    if (!moved) { status = 2; break; }
    // stagnation: the FP32 phase hands over, the polish stops at a jammed local minimum
    if (A::kId != 0 && P.stall_window > 0 && iters % P.stall_window == 0) {
      if (E > Ewin * (acc_t)(1.0 - P.stall_rel)) { status = 2; break; }
      Ewin = E;
    }
    if (P.budget_ns > 0) {
      // every block must take the same decision: block 0 reads the clock, a barrier publishes it
      if (gid == 0) G.res[2 * kPart] = (globaltimer_ns() - *P.t0 > P.budget_ns) ? 1.0 : 0.0;
      if (!grid_sync(ctl)) { status = 6; break; }
      const bool late = *(volatile double *)&G.res[2 * kPart] > 0.5;
      if (!grid_sync(ctl)) { status = 6; break; }
      if (late) { status = 6; break; }
    }
  }
  if (status < 4 && e_at != iters) {
    bool good = true;
    E = full_energy(good);
    if (!good) status = 6;
  }
  // ---- merge: scatter back to the caller's order
  for (int pos = gid; pos < n; pos += gstride) {
    const int i = perm[pos];
    const PP v = xw[pos];
    if (A::kId == 1) {
      P.x32[D.off + i] = make_float2((float)v.x, (float)v.y);
    } else {
      P.x64[D.off + i] = make_double2((double)v.x, (double)v.y);
      if (A::kId == 2) P.x32[D.off + i] = make_float2((float)v.x, (float)v.y);
    }
  }
  if (gid == 0) {
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
}

template <class A> cudaError_t coop_launch(const DescendParams &p, int q, const GridBufs &g, GridCtl *c, int grid,
                                           int block, cudaStream_t s) {
  DescendParams pp = p;
  int qq = q;
  GridBufs gg = g;
  GridCtl *cc = c;
  void *args[] = {&pp, &qq, &gg, &cc};
  return cudaLaunchCooperativeKernel((void *)descend_grid_kernel<A>, dim3(grid), dim3(block), args, 0, s);
}

// Self-test of the bounded wait: every block waits at a barrier that expects one block more than
// the grid has, so no arrival releases it; each wait must end by its time limit with the error
// flag raised.  Block 0 reports whether it saw the barrier fail and how long it waited.
__global__ void barrier_selftest_kernel(GridCtl *c, long long timeout_ns, int *failed, long long *waited) {
  const long long t0 = globaltimer_ns();
  const bool ok = grid_sync_n(c, gridDim.x + 1u, timeout_ns);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *failed = ok ? 0 : 1;
    *waited = globaltimer_ns() - t0;
  }
}

}  // namespace

cudaError_t selftest_grid_barrier(long long timeout_ns, int *failed_host, long long *waited_host) {
  GridCtl *c = nullptr;
  int *f = nullptr;
  long long *w = nullptr;
  cudaError_t e = cudaMalloc(&c, sizeof(GridCtl));
  if (e == cudaSuccess) e = cudaMalloc(&f, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(c, 0, sizeof(GridCtl));
  if (e == cudaSuccess) {
    barrier_selftest_kernel<<<4, 32>>>(c, timeout_ns, f, w);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(failed_host, f, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(waited_host, w, sizeof(long long), cudaMemcpyDeviceToHost);
  cudaFree(c);
  cudaFree(f);
  cudaFree(w);
  return e;
}

cudaError_t grid_descend_occupancy(int arith, int block, int *bps) {
  if (arith == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_grid_kernel<Arith64>, block, 0);
  if (arith == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_grid_kernel<Arith32>, block, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_grid_kernel<ArithMix>, block, 0);
}

cudaError_t launch_grid_descend(int arith, const DescendParams &p, int q, const GridBufs &g, GridCtl *c, int grid,
                                int block, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c, 0, sizeof(GridCtl), s);
  if (e != cudaSuccess) return e;
  if (arith == 0) return coop_launch<Arith64>(p, q, g, c, grid, block, s);
  if (arith == 1) return coop_launch<Arith32>(p, q, g, c, grid, block, s);
  return coop_launch<ArithMix>(p, q, g, c, grid, block, s);
}

}  // namespace pecc
