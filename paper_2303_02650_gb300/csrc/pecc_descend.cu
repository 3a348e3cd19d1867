// pecc_descend.cu -- persistent descent kernel: Algorithm GBO (Sec. 4.1) with ANM (Sec. 4.3).
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
//     ANM) and before a batch step whenever twice the largest displacement since
//     the last build plus the step cap could exceed l_cut - 2 (Verlet rule).
//   * per batch step (Eq. 8): the batch energy of Eq. 7 and its gradient, the
//     quasi-Newton direction -H g of Eq. 10 / Eq. 11 with m secant pairs, a
//     backtracking line search in place of the argmin of Eq. 9, and a secant
//     pair push when the curvature condition holds.
//
// The direction is computed in "vector-free" form (Chen, Wang, Zhou, Burges,
// "Large-scale L-BFGS using MapReduce", NIPS 2014): the two-loop recursion is
// run on the Gram matrix of the basis {s_a, y_a, g} by one warp, and the direction
// is assembled as one linear combination.  In exact arithmetic this is the
// two-loop recursion; it replaces 2m dependent block-wide dot products by one
// batched reduction per step.
#include <cfloat>

#include "pecc_internal.h"

namespace pecc {

namespace {

constexpr int KS = kMaxSlots;     // basis index of Y slot a is KS + a
constexpr int GI = 2 * kMaxSlots; // basis index of g
constexpr int NDOT = 4 * kMaxSlots + 3;

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

template <class A> struct Smem {
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  acc_t ra[32 * 2];           // reduction scratch: acc sums
  vec_t rb[32 * NDOT];        // vec sums
  vec_t rc[32 * 2];           // maxima
  acc_t oa[2];
  vec_t ob[NDOT];
  vec_t oc[2];
  vec_t gram[kBasis * kBasis];
  vec_t coef[kBasis];
  vec_t alpha[kMaxSlots];
  int ring[kMaxSlots];
  int count, stage;
  int32_t sh[40];
  int q;
  int flag;
};

// Block reduction of NA acc sums, NB vec sums and NC vec maxima.
template <class A, int NA, int NB, int NC>
__device__ __forceinline__ void reduce(Smem<A> &S, typename A::acc_t (&a)[NA], typename A::vec_t (&b)[NB],
                                       typename A::vec_t (&c)[NC]) {
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NA; ++q) { acc_t v = warp_sum(a[q]); if (lane == 0) S.ra[w * NA + q] = v; }
#pragma unroll
  for (int q = 0; q < NB; ++q) { vec_t v = warp_sum(b[q]); if (lane == 0) S.rb[w * NB + q] = v; }
#pragma unroll
  for (int q = 0; q < NC; ++q) { vec_t v = warp_max(c[q]); if (lane == 0) S.rc[w * NC + q] = v; }
  __syncthreads();
  for (int q = threadIdx.x; q < NA + NB + NC; q += blockDim.x) {
    if (q < NA) {
      acc_t s = 0; for (int u = 0; u < nw; ++u) s += S.ra[u * NA + q];
      S.oa[q] = s;
    } else if (q < NA + NB) {
      int r = q - NA; vec_t s = 0; for (int u = 0; u < nw; ++u) s += S.rb[u * NB + r];
      S.ob[r] = s;
    } else {
      int r = q - NA - NB; vec_t s = S.rc[r]; for (int u = 1; u < nw; ++u) s = max(s, S.rc[u * NC + r]);
      S.oc[r] = s;
    }
  }
  __syncthreads();
}

template <class A>
__global__ void __launch_bounds__(A::kId == 0 ? 256 : 512)
descend_kernel(DescendParams P) {
  using pos_t = typename A::pos_t;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  using sc_t = acc_t;  // per-step scalars in the arithmetic's own precision
  using PP = v2<pos_t>;
  using VV = v2<vec_t>;
  __shared__ Smem<A> S;
  const sc_t c1 = (sc_t)P.c1, step_max = (sc_t)P.step_max, two_skin = (sc_t)(2.0 * P.rebuild_disp);
  const sc_t gsum_tol = (sc_t)P.gsum_tol, curv_eps = (sc_t)P.curv_eps;
  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int mm = P.m + 1;  // physical slots

  for (;;) {
    if (tid == 0) S.q = atomicAdd(P.queue, 1);
    __syncthreads();
    const int qi = S.q;
    __syncthreads();
    if (qi >= P.num) break;
    const int q = P.order[qi];
    const InstDesc D = P.desc[q];
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
        continue;
      }
    }
    if (n == 0) {
      if (tid == 0) { O->iters = 0; O->status = 0; O->E = 0.0; if (A::kId == 1) { O->iters32 = 0; O->status32 = 0; O->E32 = 0.0; } }
      __syncthreads();
      continue;
    }

    PP *xw = (PP *)P.xw + D.off;
    PP *xb = (PP *)P.xb + D.off;
    PP *xo = (PP *)P.xo + D.off;
    VV *g = (VV *)P.g + D.off;
    VV *gt = (VV *)P.gt + D.off;
    VV *dv = (VV *)P.d + D.off;
    VV *Sv = (VV *)P.S + (int64_t)mm * D.off;
    VV *Yv = (VV *)P.Y + (int64_t)mm * D.off;
    int32_t *perm = P.perm + D.off;
    uint64_t *skey = P.skey + D.off;
    int32_t *rpb[2] = {P.rp + D.rp_off, P.rp + D.rp_off + n + 1};
    int32_t *colb[2] = {P.col + D.col_off, P.col + D.col_off + D.cap};
    uint32_t *ckey = P.ckey + D.off;
    int32_t *corder = P.corder + D.off;
    int32_t *cells = P.cells + D.cell_off;
    vec_t *gramg = (vec_t *)P.gram + D.gram_off;
    int32_t *meta = P.meta + D.meta_off;
    const int k = D.k;
    const pos_t lc2 = (pos_t)(P.l_cut * P.l_cut);

    // ---- 1. partition key and rank (stable by index)
    for (int i = tid; i < n; i += T) {
      double x, y;
      if (A::kId == 0) { double2 v = P.x64[D.off + i]; x = v.x; y = v.y; }
      else { float2 v = P.x32[D.off + i]; x = v.x; y = v.y; }
      skey[i] = sortable(part_key(x, y, P.partition));
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
      bad |= !(isfinite((double)v.x) && isfinite((double)v.y));
      xw[p] = v;
      xb[p] = v;
    }
    bad = __syncthreads_or(bad);

    int status = 3;  // max_iter unless something else ends the run
    int iters = 0, builds = 0, changes = 0, trials = 0, resets = 0, stalls = 0;
    int cur = 0, cnt = 0, len = 1;
    sc_t Dmax = 0;  // largest displacement since the last build
    acc_t E = 0;

    auto build = [&](int into) -> int {
      return cta_build_neighbors<pos_t>(xw, n, D.R, D.inv_cs, D.ncx, lc2, ckey, corder, cells, rpb[into],
                                        colb[into], D.cap, S.sh);
    };
    // ANM step (Algorithm ANM): build Gamma', compare, keep or replace; returns false on overflow
    auto anm_rebuild = [&]() -> bool {
      int alt = cur ^ 1;
      int tot = build(alt);
      if (tot > D.cap) return false;
      ++builds;
      int diff = 0;
      const int32_t *ra = rpb[alt], *rc = rpb[cur];
      for (int i = tid; i <= n; i += T) diff |= ra[i] != rc[i];
      diff = __syncthreads_or(diff);
      if (!diff) {
        const int32_t *ca = colb[alt], *cc = colb[cur];
        for (int i = tid; i < tot; i += T) diff |= ca[i] != cc[i];
        diff = __syncthreads_or(diff);
      }
      if (diff) { cur = alt; len = 1; ++changes; }
      else if (len < (1 << 30)) len *= 2;
      cnt = 0;
      for (int p = tid; p < n; p += T) xb[p] = xw[p];
      Dmax = 0;
      __syncthreads();
      return true;
    };
    // full energy (Eq. 5 over the lists: each pair from its larger index)
    auto full_energy = [&]() -> acc_t {
      const int32_t *rp = rpb[cur], *cl = colb[cur];
      acc_t a[1] = {0};
      vec_t b[1] = {0}, c[1] = {0};
      for (int p = tid; p < n; p += T) {
        PP xi = xw[p];
        acc_t e = 0;
        for (int t = rp[p]; t < rp[p + 1]; ++t) {
          int j = cl[t];
          if (j >= p) continue;
          vec_t fx, fy;
          acc_t d = A::pair(xi, xw[j], fx, fy);
          e += d * d;
        }
        vec_t fx, fy;
        acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
        a[0] += e + d0 * d0;
      }
      reduce<A, 1, 1, 1>(S, a, b, c);
      return S.oa[0];
    };

    if (bad) {
      status = 5;
    } else {
      int tot = build(0);
      if (tot > D.cap) status = 4;
      else {
        builds = 1;
        E = full_energy();
        if (!isfinite((double)E)) status = 5;
        else if (E <= (acc_t)P.e_tol) status = 0;
      }
    }
    for (int u = tid; u < k * kMetaInts; u += T) meta[u] = 0;
    for (int u = tid; u < k * kBasis * kBasis; u += T) gramg[u] = vec_t(0);
    __syncthreads();

    const int q_ = n / k, r_ = n % k;
    bool fresh = false;  // k == 1: g / E of the previous accepted trial are current
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
        const int32_t *rp = rpb[cur], *cl = colb[cur];
        // batch ring metadata and Gram block into shared memory
        if (tid == 0) {
          S.count = meta[p * kMetaInts + 0];
          S.stage = meta[p * kMetaInts + 1];
          for (int c = 0; c < kMaxSlots; ++c) S.ring[c] = meta[p * kMetaInts + 2 + c];
        }
        for (int u = tid; u < kBasis * kBasis; u += T) S.gram[u] = gramg[(size_t)p * kBasis * kBasis + u];
        __syncthreads();
        const int count = S.count;

        // ---- pass A: batch energy (Eq. 7) and gradient, dots of g with the stored pairs
        acc_t aA[1] = {0};
        vec_t bA[2 + 2 * kMaxSlots];
        vec_t cA[1] = {0};
#pragma unroll
        for (int u = 0; u < 2 + 2 * kMaxSlots; ++u) bA[u] = 0;
        if (fresh) { VV *t_ = g; g = gt; gt = t_; }
        for (int pos = b + tid; pos < e; pos += T) {
          PP xi = xw[pos];
          xo[pos] = xi;
          VV gi;
          if (!fresh) {
            vec_t gx = 0, gy = 0;
            acc_t ei = 0;
            for (int t = rp[pos]; t < rp[pos + 1]; ++t) {
              int j = cl[t];
              vec_t fx, fy;
              acc_t d = A::pair(xi, xw[j], fx, fy);
              gx += fx; gy += fy;
              if (j < b || j >= e || j < pos) ei += d * d;
            }
            vec_t fx, fy;
            acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
            gx += fx; gy += fy;
            aA[0] += ei + d0 * d0;
            gi.x = gx; gi.y = gy;
            g[pos] = gi;
          } else {
            gi = g[pos];
          }
          bA[0] += gi.x * gi.x + gi.y * gi.y;
#pragma unroll
          for (int c = 0; c < kMaxSlots; ++c) {
            if (c < count) {
              int sl = S.ring[c];
              VV s = Sv[(int64_t)sl * n + pos], y = Yv[(int64_t)sl * n + pos];
              bA[1 + c] += gi.x * s.x + gi.y * s.y;
              bA[1 + kMaxSlots + c] += gi.x * y.x + gi.y * y.y;
            }
          }
        }
        reduce<A, 1, 2 + 2 * kMaxSlots, 1>(S, aA, bA, cA);
        const acc_t Ep = fresh ? E : S.oa[0];
        const vec_t gg = S.ob[0];
        const sc_t gnorm = sqrt((sc_t)gg);
        gsum += gnorm;
        fresh = false;
        if (!(gnorm > sc_t(0))) {
          if (!isfinite(gnorm)) status = 5;
          continue;
        }

        // ---- scalar two-loop on the Gram matrix (warp 0), lane = basis index
        if (warp == 0) {
          vec_t *G = S.gram;
          if (lane < count) {
            int sl = S.ring[lane];
            G[GI * kBasis + sl] = G[sl * kBasis + GI] = S.ob[1 + lane];
            G[GI * kBasis + KS + sl] = G[(KS + sl) * kBasis + GI] = S.ob[1 + kMaxSlots + lane];
          }
          if (lane == 0) G[GI * kBasis + GI] = gg;
          __syncwarp();
          vec_t del = (lane == GI) ? vec_t(1) : vec_t(0);
          for (int c = count - 1; c >= 0; --c) {
            int sl = S.ring[c];
            vec_t prod = (lane < kBasis) ? del * G[sl * kBasis + lane] : vec_t(0);
            vec_t a = warp_sum(prod) / G[sl * kBasis + KS + sl];
            if (lane == 0) S.alpha[c] = a;
            if (lane == KS + sl) del -= a;
          }
          if (count > 0) {
            int nw_ = S.ring[count - 1];
            vec_t gam = G[nw_ * kBasis + KS + nw_] / G[(KS + nw_) * kBasis + KS + nw_];
            del *= gam;
          }
          __syncwarp();
          for (int c = 0; c < count; ++c) {
            int sl = S.ring[c];
            vec_t prod = (lane < kBasis) ? del * G[(KS + sl) * kBasis + lane] : vec_t(0);
            vec_t bb = warp_sum(prod) / G[sl * kBasis + KS + sl];
            if (lane == sl) del += S.alpha[c] - bb;
          }
          if (lane < kBasis) S.coef[lane] = -del;
        }
        __syncthreads();

        bool accepted = false;
        acc_t Et = 0;
        vec_t disp2 = 0;
        for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
          if (attempt == 1) {
            if (S.count == 0) break;
            __syncthreads();
            if (tid == 0) { S.count = 0; meta[p * kMetaInts + 0] = 0; }
            ++resets;
            for (int u = tid; u < kBasis; u += T) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
            __syncthreads();
          }
          // ---- pass B: direction, g'd and the largest per-circle move
          for (int round = 0; round < 2; ++round) {
            const int cnt_now = S.count;
            acc_t aB[1] = {0};
            vec_t bB[1] = {0}, cB[1] = {0};
            for (int pos = b + tid; pos < e; pos += T) {
              VV gi = g[pos];
              vec_t cg = S.coef[GI];
              vec_t dx = cg * gi.x, dy = cg * gi.y;
              for (int c = 0; c < cnt_now; ++c) {
                int sl = S.ring[c];
                vec_t cs = S.coef[sl], cy = S.coef[KS + sl];
                VV s = Sv[(int64_t)sl * n + pos], y = Yv[(int64_t)sl * n + pos];
                dx += cs * s.x + cy * y.x;
                dy += cs * s.y + cy * y.y;
              }
              VV dd; dd.x = dx; dd.y = dy;
              dv[pos] = dd;
              bB[0] += gi.x * dx + gi.y * dy;
              cB[0] = max(cB[0], dx * dx + dy * dy);
            }
            reduce<A, 1, 1, 1>(S, aB, bB, cB);
            if (S.ob[0] < vec_t(0) || round == 1) break;
            // not a descent direction: drop the memory, take -g
            if (tid == 0) { S.count = 0; meta[p * kMetaInts + 0] = 0; }
            if (cnt_now > 0) ++resets;
            for (int u = tid; u < kBasis; u += T) S.coef[u] = (u == GI) ? vec_t(-1) : vec_t(0);
            __syncthreads();
          }
          const sc_t gd = (sc_t)S.ob[0];
          const sc_t dmax = sqrt((sc_t)S.oc[0]);
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
            acc_t aD[1] = {0};
            vec_t bD[1] = {0}, cD[1] = {0};
            for (int pos = b + tid; pos < e; pos += T) {
              PP xi = xw[pos];
              vec_t gx = 0, gy = 0;
              acc_t ei = 0;
              for (int t = rp[pos]; t < rp[pos + 1]; ++t) {
                int j = cl[t];
                vec_t fx, fy;
                acc_t d = A::pair(xi, xw[j], fx, fy);
                gx += fx; gy += fy;
                if (j < b || j >= e || j < pos) ei += d * d;
              }
              vec_t fx, fy;
              acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
              gx += fx; gy += fy;
              aD[0] += ei + d0 * d0;
              VV gg_; gg_.x = gx; gg_.y = gy;
              gt[pos] = gg_;
              PP x0 = xb[pos];
              vec_t ex = (vec_t)(xi.x - x0.x), ey = (vec_t)(xi.y - x0.y);
              cD[0] = max(cD[0], ex * ex + ey * ey);
            }
            reduce<A, 1, 1, 1>(S, aD, bD, cD);
            ++trials;
            Et = S.oa[0];
            if (Et <= Ep + c1 * al * gd) {
              accepted = true;
              disp2 = S.oc[0];
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

        // ---- pass E: secant pair s = x_new - x_old, y = g_new - g_old and its dots
        {
          const int st = S.stage, cnt_now = S.count;
          acc_t aE[1] = {0};
          vec_t bE[NDOT];
          vec_t cE[1] = {0};
#pragma unroll
          for (int u = 0; u < NDOT; ++u) bE[u] = 0;
          for (int pos = b + tid; pos < e; pos += T) {
            PP xn = xw[pos], x0 = xo[pos];
            VV s_; s_.x = (vec_t)(xn.x - x0.x); s_.y = (vec_t)(xn.y - x0.y);
            VV gn = gt[pos], go = g[pos];
            VV y_; y_.x = gn.x - go.x; y_.y = gn.y - go.y;
            Sv[(int64_t)st * n + pos] = s_;
            Yv[(int64_t)st * n + pos] = y_;
#pragma unroll
            for (int c = 0; c < kMaxSlots; ++c) {
              if (c < cnt_now) {
                int sl = S.ring[c];
                VV s = Sv[(int64_t)sl * n + pos], y = Yv[(int64_t)sl * n + pos];
                bE[c] += s_.x * s.x + s_.y * s.y;
                bE[kMaxSlots + c] += s_.x * y.x + s_.y * y.y;
                bE[2 * kMaxSlots + c] += y_.x * s.x + y_.y * s.y;
                bE[3 * kMaxSlots + c] += y_.x * y.x + y_.y * y.y;
              }
            }
            bE[4 * kMaxSlots + 0] += s_.x * s_.x + s_.y * s_.y;
            bE[4 * kMaxSlots + 1] += s_.x * y_.x + s_.y * y_.y;
            bE[4 * kMaxSlots + 2] += y_.x * y_.x + y_.y * y_.y;
          }
          reduce<A, 1, NDOT, 1>(S, aE, bE, cE);
          const vec_t ss = S.ob[4 * kMaxSlots], sy = S.ob[4 * kMaxSlots + 1], yy = S.ob[4 * kMaxSlots + 2];
          const bool push = (sc_t)sy > curv_eps * sqrt((sc_t)ss) * sqrt((sc_t)yy) && P.m > 0;
          if (push) {
            vec_t *G = S.gram;
            if (tid < cnt_now) {
              int sl = S.ring[tid];
              G[st * kBasis + sl] = G[sl * kBasis + st] = S.ob[tid];
              G[st * kBasis + KS + sl] = G[(KS + sl) * kBasis + st] = S.ob[kMaxSlots + tid];
              G[(KS + st) * kBasis + sl] = G[sl * kBasis + KS + st] = S.ob[2 * kMaxSlots + tid];
              G[(KS + st) * kBasis + KS + sl] = G[(KS + sl) * kBasis + KS + st] = S.ob[3 * kMaxSlots + tid];
            }
            if (tid == 0) {
              G[st * kBasis + st] = ss;
              G[st * kBasis + KS + st] = G[(KS + st) * kBasis + st] = sy;
              G[(KS + st) * kBasis + KS + st] = yy;
            }
            __syncthreads();
            for (int u = tid; u < kBasis * kBasis; u += T) gramg[(size_t)p * kBasis * kBasis + u] = S.gram[u];
            if (tid == 0) {
              int c = S.count;
              if (c < P.m) {
                S.ring[c] = st;
                S.count = c + 1;
                int fr = 0;  // first slot not in the ring
                for (; fr < mm; ++fr) {
                  bool used = false;
                  for (int u = 0; u <= c; ++u) used |= (S.ring[u] == fr);
                  if (!used) break;
                }
                S.stage = fr;
              } else {
                int ev = S.ring[0];
                for (int u = 0; u + 1 < c; ++u) S.ring[u] = S.ring[u + 1];
                S.ring[c - 1] = st;
                S.stage = ev;
              }
              meta[p * kMetaInts + 0] = S.count;
              meta[p * kMetaInts + 1] = S.stage;
              for (int u = 0; u < kMaxSlots; ++u) meta[p * kMetaInts + 2 + u] = S.ring[u];
            }
            __syncthreads();
          }
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
      if (!(k == 1 && fresh)) { E = full_energy(); }
      if (!isfinite((double)E)) { status = 5; break; }
      if (E <= (acc_t)P.e_tol) { status = 0; break; }
      if (gsum <= gsum_tol) { status = 1; break; }
      if (!moved) { status = 2; break; }
      // FP32 phase: binary32 has reached its resolution when E stops falling; hand over
      if (A::kId == 1 && P.stall_window > 0 && iters % P.stall_window == 0) {
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
      O->cur = cur;
    }
    __syncthreads();
  }
}

}  // namespace

__global__ void stamp_kernel(long long *t0) { *t0 = globaltimer_ns(); }

cudaError_t launch_stamp(long long *t0, cudaStream_t s) {
  stamp_kernel<<<1, 1, 0, s>>>(t0);
  return cudaGetLastError();
}

cudaError_t launch_descend(int arith, const DescendParams &p, int grid, int block, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (arith == 0) descend_kernel<Arith64><<<grid, block, 0, s>>>(p);
  else if (arith == 1) descend_kernel<Arith32><<<grid, block, 0, s>>>(p);
  else descend_kernel<ArithMix><<<grid, block, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t descend_attributes(int arith, cudaFuncAttributes *attr) {
  if (arith == 0) return cudaFuncGetAttributes(attr, descend_kernel<Arith64>);
  if (arith == 1) return cudaFuncGetAttributes(attr, descend_kernel<Arith32>);
  return cudaFuncGetAttributes(attr, descend_kernel<ArithMix>);
}

int descend_max_block(int arith) { return arith == 0 ? 256 : 512; }

cudaError_t descend_occupancy(int arith, int block, int *bps) {
  if (arith == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_kernel<Arith64>, block, 0);
  if (arith == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_kernel<Arith32>, block, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, descend_kernel<ArithMix>, block, 0);
}

}  // namespace pecc
