// pecc_adjust.cu -- container adjustment (Sec. 4.2, Algorithm adjust_container, Eq. 12) on the GPU.
//
// z = (x, R) and U(z, lambda) = E(x, R) + lambda R^2.  For each of `rounds` rounds a limited-memory
// BFGS minimises U over all of z (one batch; a fresh memory each round), then lambda is halved.
// dU/dx is the gradient of E; dU/dR = -2 sum_i d_i0 + 2 lambda R.  One thread block per instance
// (persistent over a work queue), binary64 throughout, the two-loop recursion written out over
// the stored pairs (each dot product one block reduction in a fixed order: deterministic).  The
// lists are maintained as in the descent: a cell-list build, the Verlet rule before a step and
// ANM after each iteration.
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

__global__ void __launch_bounds__(kAdjT) adjust_kernel(AdjustParams P) {
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
    double2 *g = P.g + D.off, *gn = P.gn + D.off, *dv = P.d + D.off, *zo = P.zo + D.off;
    double2 *xb = P.xb + D.off, *xs = P.xs + D.off;
    double2 *Sv = P.S + (int64_t)kAdjM * D.off, *Yv = P.Y + (int64_t)kAdjM * D.off;
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
    auto eval = [&](double2 *gout, double Rz, double lam, double &U, double &gR) {
      const double Rm1sq = (Rz >= 1.0) ? (Rz - 1.0) * (Rz - 1.0) : -1.0;
      double v[2] = {0.0, 0.0};
      const bool mx[2] = {false, false};
      for (int i = tid; i < n; i += T) {
        const double2 xi = x[i];
        double gx = 0.0, gy = 0.0, e = 0.0;
        for (int t = rp[i]; t < rp[i + 1]; ++t) {
          const int j = col[t];
          double fx, fy;
          const double d = Arith64::pair(xi, x[j], fx, fy);
          gx += fx; gy += fy;
          if (j < i) e += d * d;
        }
        double fx, fy;
        const double d0 = Arith64::wall(xi, Rz, Rm1sq, fx, fy);
        gx += fx; gy += fy;
        v[0] += e + d0 * d0;
        v[1] += d0;
        gout[i] = make_double2(gx, gy);
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
        double v1[1] = {0.0};
        const bool mx1[1] = {false};
        for (int i = tid; i < n; i += T) { const double2 gi = g[i]; v1[0] += gi.x * gi.x + gi.y * gi.y; }
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
          for (int i = tid; i < n; i += T) dv[i] = g[i];
          double qR = gR;
          for (int c = count - 1; c >= 0; --c) {
            const int sl = (head + c) % P.m;
            const double2 *s_ = Sv + (int64_t)sl * n;
            double v[1] = {0.0};
            for (int i = tid; i < n; i += T) { const double2 a = s_[i], b = dv[i]; v[0] += a.x * b.x + a.y * b.y; }
            bred<1>(S, v, mx1);
            const double a = S.rho[sl] * (v[0] + S.sR[sl] * qR);
            if (tid == 0) S.alpha[c] = a;
            const double2 *y_ = Yv + (int64_t)sl * n;
            for (int i = tid; i < n; i += T) {
              const double2 yv = y_[i];
              double2 b = dv[i];
              b.x -= a * yv.x; b.y -= a * yv.y;
              dv[i] = b;
            }
            qR -= a * S.yR[sl];
          }
          if (count > 0) {
            const int nw_ = (head + count - 1) % P.m;
            const double gam = 1.0 / (S.rho[nw_] * S.yy[nw_]);  // s'y / y'y of the newest pair
            for (int i = tid; i < n; i += T) { double2 b = dv[i]; b.x *= gam; b.y *= gam; dv[i] = b; }
            qR *= gam;
          }
          __syncthreads();  // alpha[] written by thread 0
          for (int c = 0; c < count; ++c) {
            const int sl = (head + c) % P.m;
            const double2 *y_ = Yv + (int64_t)sl * n;
            double v[1] = {0.0};
            for (int i = tid; i < n; i += T) { const double2 a = y_[i], b = dv[i]; v[0] += a.x * b.x + a.y * b.y; }
            bred<1>(S, v, mx1);
            const double bta = S.rho[sl] * (v[0] + S.yR[sl] * qR);
            const double w = S.alpha[c] - bta;
            const double2 *s_ = Sv + (int64_t)sl * n;
            for (int i = tid; i < n; i += T) {
              const double2 sv = s_[i];
              double2 b = dv[i];
              b.x += w * sv.x; b.y += w * sv.y;
              dv[i] = b;
            }
            qR += w * S.sR[sl];
          }
          // d = -q; g'd and the largest move (circles and the radius)
          double v2[2] = {0.0, 0.0};
          const bool mx2[2] = {false, true};
          for (int i = tid; i < n; i += T) {
            double2 b = dv[i];
            b.x = -b.x; b.y = -b.y;
            dv[i] = b;
            const double2 gi = g[i];
            v2[0] += gi.x * b.x + gi.y * b.y;
            v2[1] = fmax(v2[1], b.x * b.x + b.y * b.y);
          }
          bred<2>(S, v2, mx2);
          double dR = -qR;
          double gd = v2[0] + gR * dR;
          double dmax = sqrt(fmax(v2[1], dR * dR));
          if (!(gd < 0.0)) {  // not a descent direction: drop the memory, take -g
            count = 0;
            head = 0;
            double v3[1] = {0.0};
            for (int i = tid; i < n; i += T) {
              const double2 gi = g[i];
              dv[i] = make_double2(-gi.x, -gi.y);
              v3[0] = fmax(v3[0], gi.x * gi.x + gi.y * gi.y);
            }
            const bool mx3[1] = {true};
            bred<1>(S, v3, mx3);
            dR = -gR;
            gd = -gg;
            dmax = sqrt(fmax(v3[0], dR * dR));
          }
          double al = (dmax > P.step_max) ? P.step_max / dmax : 1.0;
          for (int tr = 0; tr < P.max_trials; ++tr) {
            for (int i = tid; i < n; i += T) {
              const double2 a = zo[i], b = dv[i];
              x[i] = make_double2(a.x + al * b.x, a.y + al * b.y);
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
        // ---- the secant pair: s into zo, y into g (the new gradient is gn); displacement
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        const bool mx4[4] = {false, false, false, true};
        for (int i = tid; i < n; i += T) {
          const double2 xn = x[i], x0 = zo[i], gnew = gn[i], gold = g[i], b0 = xb[i];
          const double2 s_ = make_double2(xn.x - x0.x, xn.y - x0.y);
          const double2 y_ = make_double2(gnew.x - gold.x, gnew.y - gold.y);
          zo[i] = s_;
          g[i] = y_;
          v4[0] += s_.x * y_.x + s_.y * y_.y;
          v4[1] += s_.x * s_.x + s_.y * s_.y;
          v4[2] += y_.x * y_.x + y_.y * y_.y;
          const double ex = xn.x - b0.x, ey = xn.y - b0.y;
          v4[3] = fmax(v4[3], ex * ex + ey * ey);
        }
        bred<4>(S, v4, mx4);
        const double sR = R - Ro, yR = gnR - gR;
        const double sy = v4[0] + sR * yR, ss = v4[1] + sR * sR, yy = v4[2] + yR * yR;
        Dmax = fmax(Dmax, sqrt(v4[3]));
        if (P.m > 0 && sy > P.curv_eps * sqrt(ss) * sqrt(yy)) {
          int sl;
          if (count < P.m) { sl = (head + count) % P.m; ++count; }
          else { sl = head; head = (head + 1) % P.m; }
          double2 *s_ = Sv + (int64_t)sl * n, *y_ = Yv + (int64_t)sl * n;
          for (int i = tid; i < n; i += T) { s_[i] = zo[i]; y_[i] = g[i]; }
          if (tid == 0) { S.sR[sl] = sR; S.yR[sl] = yR; S.rho[sl] = 1.0 / sy; S.yy[sl] = yy; }
        }
        { double2 *t_ = g; g = gn; gn = t_; }  // the trial's gradient is the next iteration's
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

cudaError_t launch_adjust(const AdjustParams &p, int grid, cudaStream_t s) {
  if (p.num <= 0 || grid <= 0) return cudaSuccess;
  adjust_kernel<<<grid, kAdjT, 0, s>>>(p);
  return cudaGetLastError();
}

int adjust_max_m() { return kAdjM; }

}  // namespace pecc
