// pecc_dense.cu -- GBO with the explicit inverse Hessian of each batch (Sec. 4.1, Eq. 8, Eq. 10,
// Eq. 11): the paper's own quasi-Newton update, binary64, one thread block per instance.
//
// Each batch p of N = 2 |B_p| coordinates keeps H_p (N x N, row major, in HBM).  It starts as I,
// is rescaled to (s'y / y'y) I before its first update, and each accepted pair with enough
// curvature applies Eq. 11 as the symmetric rank-two change
//   H+ = H - rho (Hy) s' - rho s (Hy)' + (rho^2 y'Hy + rho) s s',   rho = 1 / (y's).
// A batch step costs two products with H (the direction -H g and H y) and one pass that rewrites
// H: 4 N^2 binary64 words of HBM traffic and about 5 N^2 FMA, against O(N) for the rest of the
// step.  The products run one warp per row (coalesced rows, lanes over columns).
// Everything else follows the limited-memory descent: the partition of Sec. 4.1, the Armijo
// search on the batch energy of Eq. 7 with the step cap, the Verlet rule before a batch step and
// ANM after each sweep (Algorithm ANM), and the stop tests of Algorithm GBO.
#include "pecc_internal.h"

namespace pecc {

namespace {

constexpr int kDT = 256;
constexpr int kDW = kDT / 32;

struct DSmem {
  double red[kDW][4];
  double tot[4];
  int32_t sh[40];
  int32_t fresh[kMaxK];
  unsigned long long hash;
  int q;
};

template <int NV>
__device__ __forceinline__ void dred(DSmem &S, double (&v)[NV], const bool (&mx)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const double s = mx[q] ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0) S.red[w][q] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int q = threadIdx.x;
    double s = S.red[0][q];
    for (int u = 1; u < nw; ++u) s = mx[q] ? fmax(s, S.red[u][q]) : s + S.red[u][q];
    S.tot[q] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = S.tot[q];
  __syncthreads();
}

// out[r] = sign * (H in[])[r], r < N; one warp per row.
__device__ __forceinline__ void gemv(const double *__restrict__ H, int N, const double *in, double *out,
                                     double sign) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < N; r += kDW) {
    const double *h = H + (int64_t)r * N;
    double v = 0.0;
    for (int c = lane; c < N; c += 32) v = fma(h[c], in[c], v);
    v = warp_sum(v);
    if (lane == 0) out[r] = sign * v;
  }
}

__global__ void __launch_bounds__(kDT, 2) dense_kernel(DenseParams P) {
  __shared__ DSmem S;
  const int tid = threadIdx.x, T = blockDim.x;
  const double lc2 = P.l_cut * P.l_cut;
  for (;;) {
    if (tid == 0) S.q = atomicAdd(P.queue, 1);
    __syncthreads();
    const int qi = S.q;
    __syncthreads();
    if (qi >= P.num) break;
    const int q = P.order[qi];
    const InstDesc D = P.desc[q];
    const int n = D.n;
    InstOut *O = P.out + q;
    if (n == 0) {
      if (tid == 0) { O->iters = 0; O->status = 0; O->E = 0.0; O->iters32 = 0; O->trials32 = 0; }
      __syncthreads();
      continue;
    }
    const int k = min(D.k, n);
    double2 *x = P.x + D.off;
    double2 *g = P.g + D.off, *gn = P.gn + D.off, *dv = P.d + D.off, *xo = P.xo + D.off;
    double2 *xb = P.xb + D.off, *xs = P.xs + D.off;
    double *hy = (double *)(P.hy + D.off);
    uint64_t *skey = P.skey + D.off;
    int32_t *perm = P.perm + D.off, *batch_of = P.batch_of + D.off;
    int32_t *rp = P.rp + D.rp_off, *col = P.col + D.col_off;
    const int cap = 2 * D.cap;
    uint32_t *ckey = P.ckey + D.off;
    int32_t *corder = P.corder + D.off, *cells = P.cells + D.cell_off;
    double *Hq = P.H + P.h_off[q];
    const CellGrid G{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
    const double R = D.R, Rm1sq = (R >= 1.0) ? (R - 1.0) * (R - 1.0) : -1.0;
    const int nq = n / k, nr = n % k;
    auto bstart = [&](int p) { return p * nq + min(p, nr); };
    auto hoff = [&](int p) {  // sum of (2 |B_t|)^2 over t < p
      int64_t o = 0;
      for (int t = 0; t < p; ++t) { const int64_t m = 2 * (nq + (t < nr)); o += m * m; }
      return o;
    };

    // ---- partition (Sec. 4.1): keys, rank by (key, index), batch of every circle
    for (int i = tid; i < n; i += T) {
      const double2 v = x[i];
      skey[i] = sortable(P.partition == 3 ? random_part_key(P.part_seed, i, q) : part_key(v.x, v.y, P.partition));
    }
    __syncthreads();
    for (int i = tid; i < n; i += T) {
      const uint64_t ki = skey[i];
      int r = 0;
      for (int j = 0; j < n; ++j) {
        const uint64_t kj = skey[j];
        r += (kj < ki) || (kj == ki && j < i);
      }
      perm[r] = i;
    }
    __syncthreads();
    for (int r = tid; r < n; r += T) {
      const int p = (r < nr * (nq + 1)) ? r / (nq + 1) : nr + (r - nr * (nq + 1)) / max(nq, 1);
      batch_of[perm[r]] = p;
    }
    // ---- H_p = I for every batch
    if (tid < k) S.fresh[tid] = 1;
    for (int p = 0; p < k; ++p) {
      const int N = 2 * (nq + (p < nr));
      double *H = Hq + hoff(p);
      for (int64_t e = tid; e < (int64_t)N * N; e += T) H[e] = (e / N == e % N) ? 1.0 : 0.0;
    }
    __syncthreads();

    int status = 3, builds = 0, trials = 0, resets = 0, stalls = 0, cnt = 0, len = 1, t = 0;
    unsigned long long hcur = 0ull;
    double Dmax = 0.0;
    bool ok = true;
    auto rebuild = [&](bool anm) -> bool {
      const int tot = cta_build_neighbors<double, int32_t>(x, n, G, lc2, ckey, corder, cells, xs, rp, col, cap, S.sh,
                                                          &S.hash, false);
      ++builds;
      if (tot > cap) return false;
      if (anm) {
        const unsigned long long h = S.hash;
        if (h != hcur) { hcur = h; len = 1; }
        else if (len < (1 << 30)) len *= 2;
        cnt = 0;
      } else {
        hcur = S.hash;
      }
      for (int i = tid; i < n; i += T) xb[i] = x[i];
      Dmax = 0.0;
      __syncthreads();
      return true;
    };
    // energy of the whole instance (Eq. 5)
    auto energy = [&]() {
      double v[1] = {0.0};
      const bool mx[1] = {false};
      for (int i = tid; i < n; i += T) {
        const double2 xi = x[i];
        double fx, fy;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
          const int j = col[e];
          if (j < i) { const double d = Arith64::pair(xi, x[j], fx, fy); v[0] += d * d; }
        }
        const double d0 = Arith64::wall(xi, R, Rm1sq, fx, fy);
        v[0] += d0 * d0;
      }
      dred<1>(S, v, mx);
      return v[0];
    };
    // batch energy of Eq. 7 over the members mb[0..nb)
    auto benergy = [&](const int32_t *mb, int nb, int p) {
      double v[1] = {0.0};
      const bool mx[1] = {false};
      for (int a = tid; a < nb; a += T) {
        const int i = mb[a];
        const double2 xi = x[i];
        double fx, fy;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
          const int j = col[e];
          if (batch_of[j] == p && j >= i) continue;
          const double d = Arith64::pair(xi, x[j], fx, fy);
          v[0] += d * d;
        }
        const double d0 = Arith64::wall(xi, R, Rm1sq, fx, fy);
        v[0] += d0 * d0;
      }
      dred<1>(S, v, mx);
      return v[0];
    };
    // gradient rows of the members, in batch order
    auto bgrad = [&](const int32_t *mb, int nb, double2 *out) {
      for (int a = tid; a < nb; a += T) {
        const int i = mb[a];
        const double2 xi = x[i];
        double gx = 0.0, gy = 0.0, fx, fy;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
          Arith64::pair(xi, x[col[e]], fx, fy);
          gx += fx; gy += fy;
        }
        Arith64::wall(xi, R, Rm1sq, fx, fy);
        out[a] = make_double2(gx + fx, gy + fy);
      }
    };

    ok = rebuild(false);
    double E = ok ? energy() : 0.0;
    if (!ok) status = 4;
    else if (E <= P.e_tol) status = 0;
    while (ok && status != 0 && t < P.max_iter) {
      ++t;
      double gsum = 0.0;
      bool moved = false;
      for (int p = 0; p < k && ok; ++p) {
        if (2.0 * Dmax + P.step_max > 2.0 * P.rebuild_disp) {
          if (!rebuild(true)) { ok = false; break; }
        }
        const int32_t *mb = perm + bstart(p);
        const int nb = nq + (p < nr), N = 2 * nb;
        double *H = Hq + hoff(p);
        const double E0 = benergy(mb, nb, p);
        bgrad(mb, nb, g);
        for (int a = tid; a < nb; a += T) xo[a] = x[mb[a]];
        double v1[1] = {0.0};
        const bool mx1[1] = {false};
        for (int a = tid; a < nb; a += T) { const double2 ga = g[a]; v1[0] += ga.x * ga.x + ga.y * ga.y; }
        dred<1>(S, v1, mx1);  // also orders g and xo before the products below
        const double gnorm = sqrt(v1[0]);
        gsum += gnorm;
        if (gnorm == 0.0) continue;
        bool accepted = false;
        double gd = 0.0;
        for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
          if (attempt == 1) {
            if (S.fresh[p]) break;
            for (int64_t e = tid; e < (int64_t)N * N; e += T) H[e] = (e / N == e % N) ? 1.0 : 0.0;
            __syncthreads();
            if (tid == 0) S.fresh[p] = 1;
            ++resets;
            __syncthreads();
          }
          gemv(H, N, (const double *)g, (double *)dv, -1.0);
          __syncthreads();
          double v2[1] = {0.0};
          for (int a = tid; a < nb; a += T) { const double2 ga = g[a], da = dv[a]; v2[0] += ga.x * da.x + ga.y * da.y; }
          dred<1>(S, v2, mx1);
          gd = v2[0];
          if (!(gd < 0.0)) {  // not a descent direction: back to I and the gradient step
            if (!S.fresh[p]) {
              for (int64_t e = tid; e < (int64_t)N * N; e += T) H[e] = (e / N == e % N) ? 1.0 : 0.0;
              __syncthreads();
              if (tid == 0) S.fresh[p] = 1;
              ++resets;
            }
            for (int a = tid; a < nb; a += T) { const double2 ga = g[a]; dv[a] = make_double2(-ga.x, -ga.y); }
            gd = -gnorm * gnorm;
            __syncthreads();
          }
          double v3[1] = {0.0};
          const bool mx3[1] = {true};
          for (int a = tid; a < nb; a += T) { const double2 da = dv[a]; v3[0] = fmax(v3[0], da.x * da.x + da.y * da.y); }
          dred<1>(S, v3, mx3);
          const double dmax = sqrt(v3[0]);
          double al = (dmax > P.step_max) ? P.step_max / dmax : 1.0;
          for (int tr = 0; tr < P.max_trials; ++tr) {
            for (int a = tid; a < nb; a += T) {
              const double2 o = xo[a], da = dv[a];
              x[mb[a]] = make_double2(o.x + al * da.x, o.y + al * da.y);
            }
            __syncthreads();
            ++trials;
            const double Et = benergy(mb, nb, p);
            if (Et <= E0 + P.c1 * al * gd) { accepted = true; break; }
            al *= 0.5;
          }
          if (!accepted) {
            for (int a = tid; a < nb; a += T) x[mb[a]] = xo[a];
            __syncthreads();
          }
        }
        if (!accepted) { ++stalls; continue; }
        moved = true;
        bgrad(mb, nb, gn);
        __syncthreads();
        // s into xo, y into g; displacement since the last build
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        const bool mx4[4] = {false, false, false, true};
        for (int a = tid; a < nb; a += T) {
          const int i = mb[a];
          const double2 xn = x[i], o = xo[a], gnew = gn[a], gold = g[a], b0 = xb[i];
          const double2 s_ = make_double2(xn.x - o.x, xn.y - o.y), y_ = make_double2(gnew.x - gold.x, gnew.y - gold.y);
          xo[a] = s_;
          g[a] = y_;
          v4[0] += s_.x * y_.x + s_.y * y_.y;
          v4[1] += s_.x * s_.x + s_.y * s_.y;
          v4[2] += y_.x * y_.x + y_.y * y_.y;
          const double ex = xn.x - b0.x, ey = xn.y - b0.y;
          v4[3] = fmax(v4[3], ex * ex + ey * ey);
        }
        dred<4>(S, v4, mx4);
        Dmax = fmax(Dmax, sqrt(v4[3]));
        const double sy = v4[0], ss = v4[1], yy = v4[2];
        if (sy > P.curv_eps * sqrt(ss) * sqrt(yy)) {
          if (S.fresh[p]) {
            const double gam = sy / yy;
            for (int64_t e = tid; e < (int64_t)N * N; e += T) H[e] = (e / N == e % N) ? gam : 0.0;
            __syncthreads();
            if (tid == 0) S.fresh[p] = 0;
          }
          const double *sv = (const double *)xo, *yv = (const double *)g;
          gemv(H, N, yv, hy, 1.0);
          __syncthreads();
          double v5[1] = {0.0};
          for (int c = tid; c < N; c += T) v5[0] += yv[c] * hy[c];
          dred<1>(S, v5, mx1);
          const double rho = 1.0 / sy, cs = rho * rho * v5[0] + rho;
          const int lane = tid & 31, w = tid >> 5;
          for (int r = w; r < N; r += kDW) {
            double *h = H + (int64_t)r * N;
            const double sr = sv[r], hr = hy[r];
            for (int c = lane; c < N; c += 32) h[c] += -rho * (hr * sv[c] + sr * hy[c]) + cs * sr * sv[c];
          }
          __syncthreads();
        }
      }
      if (!ok) break;
      if (P.anm) {
        ++cnt;
        if (cnt >= len && !rebuild(true)) { ok = false; break; }
      }
      E = energy();
      if (E <= P.e_tol) status = 0;
      else if (gsum <= P.gsum_tol) { status = 1; break; }
      else if (!moved) { status = 2; break; }
    }
    if (!ok) status = 4;
    if (tid == 0) {
      O->iters = t; O->status = status; O->E = E; O->builds = builds; O->trials = trials;
      O->resets = resets; O->stalls = stalls; O->polished = 0;
      O->iters32 = t; O->status32 = status; O->trials32 = trials;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_dense(const DenseParams &p, int grid, cudaStream_t s) {
  if (p.num <= 0 || grid <= 0) return cudaSuccess;
  dense_kernel<<<grid, kDT, 0, s>>>(p);
  return cudaGetLastError();
}

// Binary64 words of the inverse Hessians of an instance of n circles in k batches.
int64_t dense_h_words(int n, int k) {
  if (n <= 0) return 0;
  k = std::max(1, std::min(k, n));
  const int64_t nq = n / k, nr = n % k;
  int64_t w = 0;
  for (int p = 0; p < k; ++p) { const int64_t m = 2 * (nq + (p < nr)); w += m * m; }
  return w;
}

}  // namespace pecc
