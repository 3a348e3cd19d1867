// pecc_adjust.cu -- container adjustment (Sec. 4.2, Algorithm adjust_container, Eq. 12) on the GPU.
//
// z = (x, R) and U(z, lambda) = E(x, R) + lambda R^2.  For each of `rounds` rounds a limited-memory
// BFGS minimises U over all of z (one batch; a fresh memory each round), then lambda is halved.
// dU/dx is the gradient of E; dU/dR = -2 sum_i d_i0 + 2 lambda R.  One thread block per instance
// (persistent over a work queue), the two-loop recursion written out over the stored pairs (each
// dot product one block reduction in a fixed order: deterministic).  The lists are maintained as
// in the descent: a cell-list build, the Verlet rule before a step and ANM after each iteration.
// Two arithmetic forms:
//   <Arith64, double>  binary64 throughout (the binary64 contexts);
//   <ArithMix, float>  the descent's polish arithmetic for the pair and wall terms (binary64
//                      coordinates, differences and the near-contact quantities 4 - l^2 and
//                      |c|^2 - (R - 1)^2, binary32 depths and forces), binary32 gradients and
//                      quasi-Newton vectors, binary64 energy sums and everything about R.
// GB300 issues few binary64 operations per clock; in the binary64 form the pair terms and the
// two-loop recursion keep that pipe about 80 % busy.  The binary32 depths put a relative jitter of
// about 1e-7 on E, so the Armijo test on U resolves U's minimum only to about 1e-6 of R while E is
// large (a large lambda); the schedule's late rounds, where the radius is settled, have E near 0.
#include "pecc_internal.h"

namespace pecc {

namespace {

constexpr int kAdjT = 256;  // threads per instance block
constexpr int kAdjW = kAdjT / 32;
constexpr int kAdjM = kMaxSlots - 1;  // memory pairs at most

struct AdjSmem {
  double red[kAdjW][4];
  double tot[4];
  double sR[kAdjM], yR[kAdjM], rho[kAdjM], yy[kAdjM], alpha[kAdjM];
  int32_t sh[40];
  unsigned long long hash;
  int q;
};

// Block reduction of NV values (sum, or max where mx[q]); every thread gets the totals in v.
template <int NV>
__device__ __forceinline__ void bred(AdjSmem &S, double (&v)[NV], const bool (&mx)[NV]) {
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

template <class A, typename VT>
__global__ void __launch_bounds__(kAdjT) adjust_kernel(AdjustParams P) {
  using V2 = v2<VT>;
  using GT = typename A::vec_t;  // the forces' and the stored gradient's type
  using GV2 = v2<GT>;
  __shared__ AdjSmem S;
  const int tid = threadIdx.x, T = blockDim.x;
  const double lc2 = P.l_cut * P.l_cut;
  for (;;) {
    if (tid == 0) S.q = atomicAdd(P.queue, 1);
    __syncthreads();
    const int q = S.q;
    __syncthreads();
    if (q >= P.num) break;
    const InstDesc D = P.desc[q];
    const int n = D.n;
    double R = P.R[q];
    double2 *x = P.x64 + D.off;
    if (n == 0 || D.big) {
      if (tid == 0) {
        P.iters[q] = 0; P.status[q] = n == 0 ? 0 : 4;
        if (P.stats) { P.stats[2 * q] = 0; P.stats[2 * q + 1] = 0; }
      }
      __syncthreads();
      continue;
    }
    if (P.from32)
      for (int i = tid; i < n; i += T) { const float2 f = P.x32[D.off + i]; x[i] = make_double2(f.x, f.y); }
    // gradients in the forces' type, the direction and the pairs in VT (the buffers are sized for
    // double2)
    GV2 *g = (GV2 *)(P.g + D.off), *gn = (GV2 *)(P.gn + D.off);
    V2 *dv = (V2 *)(P.d + D.off), *sv = (V2 *)(P.sv + D.off);
    double2 *zo = P.zo + D.off, *xb = P.xb + D.off, *xs = P.xs + D.off;
    V2 *Sv = (V2 *)(P.S + (int64_t)kAdjM * D.off), *Yv = (V2 *)(P.Y + (int64_t)kAdjM * D.off);
    int32_t *rp = P.rp + D.rp_off, *col = P.col + D.col_off;
    const int cap = 2 * D.cap;
    const CellGrid G{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
    uint32_t *ckey = P.ckey + D.off;
    int32_t *corder = P.corder + D.off, *cells = P.cells + D.cell_off;

    int status = 3, iters = 0, cnt = 0, len = 1, trials = 0, visits = 0;
    unsigned long long hcur = 0ull;
    double Dmax = 0.0;
    // list build with ANM bookkeeping; false on a capacity overflow
    auto rebuild = [&](bool anm) -> bool {
      const int tot = cta_build_neighbors<double, int32_t>(x, n, G, lc2, ckey, corder, cells, xs, rp, col, cap, S.sh,
                                                          &S.hash, false);
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
    // U, its gradient over x into gout, and dU/dR, at the current x and radius Rz
    auto eval = [&](GV2 *gout, double Rz, double lam, double &U, double &gR) {
      const double Rm1sq = (Rz >= 1.0) ? (Rz - 1.0) * (Rz - 1.0) : -1.0;
      double v[2] = {0.0, 0.0};
      const bool mx[2] = {false, false};
      for (int i = tid; i < n; i += T) {
        const double2 xi = x[i];
        GT gx = 0, gy = 0;
        double e = 0.0;
        // two entries per step (both coordinate loads in flight); the sums take the entries in row order
        const int t1 = rp[i + 1];
        for (int t = rp[i]; t < t1; t += 2) {
          const bool two = t + 1 < t1;
          const int j1 = col[t];
          const int j2 = two ? col[t + 1] : j1;
          const double2 x1 = x[j1], x2 = x[j2];
          GT fx, fy;
          const double d1 = A::pair(xi, x1, fx, fy);
          gx += fx; gy += fy;
          if (j1 < i) e += d1 * d1;
          if (two) {
            const double d2 = A::pair(xi, x2, fx, fy);
            gx += fx; gy += fy;
            if (j2 < i) e += d2 * d2;
          }
        }
        GT fx, fy;
        const double d0 = A::wall(xi, Rz, Rm1sq, fx, fy);
        gx += fx; gy += fy;
        v[0] += e + d0 * d0;
        v[1] += d0;
        gout[i] = mk2<GT>(gx, gy);
      }
      bred<2>(S, v, mx);
      U = v[0] + lam * Rz * Rz;
      gR = -2.0 * v[1] + 2.0 * lam * Rz;
    };

    bool ok = rebuild(false);
    if (!ok) status = 4;
    double lam = P.lambda0;
    for (int round = 0; round < P.rounds && ok; ++round) {
      int head = 0, count = 0;
      double U0, gR;
      eval(g, R, lam, U0, gR);
      status = 3;
      for (int it = 0; it < P.max_iter; ++it) {
        if (2.0 * Dmax + P.step_max > 2.0 * P.rebuild_disp) {
          if (!rebuild(true)) { ok = false; status = 4; break; }
        }
        ++iters;
        const bool mx1[1] = {false};
        GT p1 = 0;
        for (int i = tid; i < n; i += T) { const GV2 gi = g[i]; p1 += gi.x * gi.x + gi.y * gi.y; }
        double v1[1] = {(double)p1};
        bred<1>(S, v1, mx1);
        const double gg = v1[0] + gR * gR, gnorm = sqrt(gg);
        if (!(gnorm > P.gsum_tol)) { status = 1; break; }
        for (int i = tid; i < n; i += T) zo[i] = x[i];
        const double Ro = R;
        bool accepted = false;
        double Ut = U0, gnR = gR;
        for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
          if (attempt == 1) {
            if (count == 0) break;
            count = 0;
            head = 0;
          }
          // ---- two-loop recursion (Nocedal & Wright, Alg. 7.4) over the stored pairs; q in dv
          visits += count;
          for (int i = tid; i < n; i += T) { const GV2 gi = g[i]; dv[i] = mk2<VT>((VT)gi.x, (VT)gi.y); }
          double qR = gR;
          for (int c = count - 1; c >= 0; --c) {
            const int sl = (head + c) % P.m;
            const V2 *s_ = Sv + (int64_t)sl * n;
            VT pv = 0;
            for (int i = tid; i < n; i += T) { const V2 a = s_[i], b = dv[i]; pv += a.x * b.x + a.y * b.y; }
            double v[1] = {(double)pv};
            bred<1>(S, v, mx1);
            const double a = S.rho[sl] * (v[0] + S.sR[sl] * qR);
            if (tid == 0) S.alpha[c] = a;
            const V2 *y_ = Yv + (int64_t)sl * n;
            const VT av = (VT)a;
            for (int i = tid; i < n; i += T) {
              const V2 yv = y_[i];
              V2 b = dv[i];
              b.x -= av * yv.x; b.y -= av * yv.y;
              dv[i] = b;
            }
            qR -= a * S.yR[sl];
          }
          if (count > 0) {
            const int nw_ = (head + count - 1) % P.m;
            const double gam = 1.0 / (S.rho[nw_] * S.yy[nw_]);  // s'y / y'y of the newest pair
            const VT gv = (VT)gam;
            for (int i = tid; i < n; i += T) { V2 b = dv[i]; b.x *= gv; b.y *= gv; dv[i] = b; }
            qR *= gam;
          }
          __syncthreads();  // alpha[] written by thread 0
          for (int c = 0; c < count; ++c) {
            const int sl = (head + c) % P.m;
            const V2 *y_ = Yv + (int64_t)sl * n;
            VT pv = 0;
            for (int i = tid; i < n; i += T) { const V2 a = y_[i], b = dv[i]; pv += a.x * b.x + a.y * b.y; }
            double v[1] = {(double)pv};
            bred<1>(S, v, mx1);
            const double bta = S.rho[sl] * (v[0] + S.yR[sl] * qR);
            const double w = S.alpha[c] - bta;
            const V2 *s_ = Sv + (int64_t)sl * n;
            const VT wv = (VT)w;
            for (int i = tid; i < n; i += T) {
              const V2 sa = s_[i];
              V2 b = dv[i];
              b.x += wv * sa.x; b.y += wv * sa.y;
              dv[i] = b;
            }
            qR += w * S.sR[sl];
          }
          // d = -q; g'd and the largest move (circles and the radius)
          const bool mx2[2] = {false, true};
          GT p2 = 0;
          VT m2 = 0;
          for (int i = tid; i < n; i += T) {
            V2 b = dv[i];
            b.x = -b.x; b.y = -b.y;
            dv[i] = b;
            const GV2 gi = g[i];
            p2 += gi.x * (GT)b.x + gi.y * (GT)b.y;
            m2 = max(m2, b.x * b.x + b.y * b.y);
          }
          double v2[2] = {(double)p2, (double)m2};
          bred<2>(S, v2, mx2);
          double dR = -qR;
          double gd = v2[0] + gR * dR;
          double dmax = sqrt(fmax(v2[1], dR * dR));
          if (!(gd < 0.0)) {  // not a descent direction: drop the memory, take -g
            count = 0;
            head = 0;
            GT m3 = 0;
            for (int i = tid; i < n; i += T) {
              const GV2 gi = g[i];
              dv[i] = mk2<VT>((VT)-gi.x, (VT)-gi.y);
              m3 = max(m3, gi.x * gi.x + gi.y * gi.y);
            }
            double v3[1] = {(double)m3};
            const bool mx3[1] = {true};
            bred<1>(S, v3, mx3);
            dR = -gR;
            gd = -gg;
            dmax = sqrt(fmax(v3[0], dR * dR));
          }
          double al = (dmax > P.step_max) ? P.step_max / dmax : 1.0;
          for (int tr = 0; tr < P.max_trials; ++tr) {
            for (int i = tid; i < n; i += T) {
              const double2 a = zo[i];
              const V2 b = dv[i];
              x[i] = make_double2(a.x + al * (double)b.x, a.y + al * (double)b.y);
            }
            R = Ro + al * dR;
            __syncthreads();
            ++trials;
            eval(gn, R, lam, Ut, gnR);
            if (Ut <= U0 + P.c1 * al * gd) { accepted = true; break; }
            al *= 0.5;
          }
          if (!accepted) {
            for (int i = tid; i < n; i += T) x[i] = zo[i];
            R = Ro;
            __syncthreads();
          }
        }
        if (!accepted) { status = 2; break; }
        // ---- the secant pair: s into sv, y into dv (the new gradient is gn); displacement
        const bool mx4[4] = {false, false, false, true};
        VT p40 = 0, p41 = 0, p42 = 0;
        double m43 = 0.0;
        for (int i = tid; i < n; i += T) {
          const double2 xn = x[i], x0 = zo[i], b0 = xb[i];
          const GV2 gnew = gn[i], gold = g[i];
          const V2 s_ = mk2<VT>((VT)(xn.x - x0.x), (VT)(xn.y - x0.y));
          const V2 y_ = mk2<VT>((VT)(gnew.x - gold.x), (VT)(gnew.y - gold.y));
          sv[i] = s_;
          dv[i] = y_;
          p40 += s_.x * y_.x + s_.y * y_.y;
          p41 += s_.x * s_.x + s_.y * s_.y;
          p42 += y_.x * y_.x + y_.y * y_.y;
          const double ex = xn.x - b0.x, ey = xn.y - b0.y;
          m43 = fmax(m43, ex * ex + ey * ey);
        }
        double v4[4] = {(double)p40, (double)p41, (double)p42, m43};
        bred<4>(S, v4, mx4);
        const double sR = R - Ro, yR = gnR - gR;
        const double sy = v4[0] + sR * yR, ss = v4[1] + sR * sR, yy = v4[2] + yR * yR;
        Dmax = fmax(Dmax, sqrt(v4[3]));
        if (P.m > 0 && sy > P.curv_eps * sqrt(ss) * sqrt(yy)) {
          int sl;
          if (count < P.m) { sl = (head + count) % P.m; ++count; }
          else { sl = head; head = (head + 1) % P.m; }
          V2 *s_ = Sv + (int64_t)sl * n, *y_ = Yv + (int64_t)sl * n;
          for (int i = tid; i < n; i += T) { s_[i] = sv[i]; y_[i] = dv[i]; }
          if (tid == 0) { S.sR[sl] = sR; S.yR[sl] = yR; S.rho[sl] = 1.0 / sy; S.yy[sl] = yy; }
        }
        { GV2 *t_ = g; g = gn; gn = t_; }  // the trial's gradient is the next iteration's
        U0 = Ut;
        gR = gnR;
        __syncthreads();
        if (P.anm) {
          ++cnt;
          if (cnt >= len && !rebuild(true)) { ok = false; status = 4; break; }
        }
      }
      lam *= 0.5;
    }
    // the adjusted layout: binary64 and its binary32 copy
    for (int i = tid; i < n; i += T) {
      const double2 v = x[i];
      if (P.x32) P.x32[D.off + i] = make_float2((float)v.x, (float)v.y);
    }
    if (tid == 0) {
      P.R[q] = R; P.iters[q] = iters; P.status[q] = status;
      if (P.stats) { P.stats[2 * q] = trials; P.stats[2 * q + 1] = visits; }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_adjust(const AdjustParams &p, int mixed, int grid, cudaStream_t s) {
  if (p.num <= 0 || grid <= 0) return cudaSuccess;
  if (mixed) adjust_kernel<ArithMix, float><<<grid, kAdjT, 0, s>>>(p);
  else adjust_kernel<Arith64, double><<<grid, kAdjT, 0, s>>>(p);
  return cudaGetLastError();
}

int adjust_max_m() { return kAdjM; }

}  // namespace pecc
