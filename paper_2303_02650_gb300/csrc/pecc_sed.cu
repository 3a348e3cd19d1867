// pecc_sed.cu -- the solution-space exploring and descent heuristic (Sec. 5.2, Algorithm SED, the
// select operator of Eq. 18) over a batch of instances.
//
// Every instance q owns M candidate slots in a descent context (slot q*M + j holds n_q circles).
// One SED iteration is three stream-ordered steps, none of which waits for the host:
//   prepare  m_q = max(1, J(E(x_q))) (capped at M; 0 once instance q is done), and the
//            perturbations x_q + r of Sec. 5.2 written into slots q*M .. q*M + m_q - 1;
//   list     the active slots in the processing order (largest instances first) and their count,
//            which the descent kernels read from device memory;
//   descent  GBO of every active slot (the context's own descent);
//   select   Eq. 18 per instance: the least candidate energy if it is below E(x_q), otherwise a
//            draw with probabilities softmax(J); the chosen candidate becomes x_q, and x*_q when
//            it lowers E(x*_q); done once E(x*_q) <= e_feas.
// Random numbers: Philox4x32-10 keyed by the seed; candidate j of iteration it draws counter
// (i, it, q, 2^31 + j) for circle i, the select draw counter (0, it, q, 2^30), the initial layout
// (i, attempt, q, 0) as the context's random initialisation does.
#include "pecc_internal.h"

namespace pecc {

namespace {

constexpr int kSedT = 256;

// J(E) = ceil(-log10 E) of Sec. 5.2; 2^30 for E <= 0 (that instance is already done).
__device__ __forceinline__ int sed_J(double E) {
  if (!(E > 0.0)) return 1 << 30;
  return (int)ceil(-log10(E));
}

__device__ __forceinline__ double sym_uniform(double amp, uint32_t hi, uint32_t lo) {
  return __dmul_rn(amp, __dsub_rn(__dmul_rn(2.0, u53(hi, lo)), 1.0));
}

// The random solution of instance q (Sec. 5.1) into the operated layout: uniform in the disk of
// radius R - 1 by rejection (mode 0), or the paper's square U(-R, R)^2 (mode 1).
__global__ void __launch_bounds__(kSedT) sed_init_kernel(SedParams P) {
  const int q = blockIdx.x;
  const int n = P.n[q];
  const double R = P.R[q], rr = R - 1.0;
  const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  double2 *x = P.x + P.off[q];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double cx = 0.0, cy = 0.0;
    if (P.init_mode == 1) {
      uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, (uint32_t)q, 0u), key);
      cx = sym_uniform(R, w.x, w.y);
      cy = sym_uniform(R, w.z, w.w);
    } else if (rr > 0.0) {
      for (uint32_t a = 0; a < 64u; ++a) {
        uint4 w = philox4x32_10(make_uint4((uint32_t)i, a, (uint32_t)q, 0u), key);
        const double tx = sym_uniform(rr, w.x, w.y), ty = sym_uniform(rr, w.z, w.w);
        if (__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)) <= __dmul_rn(rr, rr)) { cx = tx; cy = ty; break; }
      }
    }
    x[i] = make_double2(cx, cy);
  }
}

// start != 0: copy x_q unperturbed into slot q*M (the initial descent of Algorithm SED).
__global__ void __launch_bounds__(kSedT) sed_prepare_kernel(SedParams P, int start) {
  const int q = blockIdx.x;
  const int n = P.n[q];
  int m;
  if (start) {
    m = 1;
  } else if (P.Eb[q] <= P.e_feas) {  // the loop head of Algorithm SED: stop once E(x*) <= e_feas
    m = 0;
  } else {
    const int J = sed_J(P.Ex[q]);
    m = J < 1 ? 1 : (J > P.M ? P.M : J);
  }
  if (threadIdx.x == 0) P.m[q] = m;
  const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  const double2 *x = P.x + P.off[q];
  for (int j = 0; j < m; ++j) {
    const int64_t co = P.cdesc[(int64_t)q * P.M + j].off;
    double2 *c64 = P.c64 + co;
    float2 *c32 = P.c32 ? P.c32 + co : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = x[i];
      double2 o = v;
      if (!start) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)P.it, (uint32_t)q, 0x80000000u | (uint32_t)j), key);
        const double rx = sym_uniform(P.amp, w.x, w.y);
        const double ry = P.shared_r ? rx : sym_uniform(P.amp, w.z, w.w);
        o = make_double2(__dadd_rn(v.x, rx), __dadd_rn(v.y, ry));
      }
      c64[i] = o;
      if (c32) c32[i] = make_float2((float)o.x, (float)o.y);
    }
  }
}

// The active slots in the processing order and their count (one block; inclusive scan of m).
__global__ void __launch_bounds__(1024) sed_list_kernel(SedParams P) {
  __shared__ int32_t sh[40];
  __shared__ int32_t act;
  const int T = blockDim.x, t = threadIdx.x;
  if (t == 0) act = 0;
  __syncthreads();
  int a = 0;
  for (int r = t; r < P.num; r += T) {
    const int m = P.m[P.porder[r]];
    P.scan[r] = m;
    a += m > 0;
  }
  if (a) atomicAdd(&act, a);
  __syncthreads();
  block_scan_inplace(P.scan, P.num, sh);
  __syncthreads();
  for (int r = t; r < P.num; r += T) {
    const int q = P.porder[r];
    const int m = P.m[q];
    const int s0 = r == 0 ? 0 : P.scan[r - 1];
    for (int j = 0; j < m; ++j) P.list[s0 + j] = q * P.M + j;
  }
  if (t == 0) {
    *P.count = P.num > 0 ? P.scan[P.num - 1] : 0;
    *P.active = act;
    *P.left = 0;
  }
}

// Eq. 18 and the record of Algorithm SED.  Ecand: candidate energies by slot, or null for the
// descent's own results.  start != 0: the initial descent's result becomes x, x* and E(x), E(x*).
__global__ void __launch_bounds__(kSedT) sed_select_kernel(SedParams P, const double *Ecand, int start) {
  const int q = blockIdx.x;
  const int m = P.m[q];
  if (m == 0) return;  // done before this iteration
  __shared__ int s_sel, s_better;
  if (threadIdx.x == 0) {
    const int64_t s0 = (int64_t)q * P.M;
    auto E = [&](int j) { return Ecand ? Ecand[s0 + j] : P.cout[s0 + j].E; };
    int sel = 0;
    const double Ex = P.Ex[q];
    if (!start && m > 1) {
      int best = 0;
      for (int j = 1; j < m; ++j)
        if (E(j) < E(best)) best = j;
      if (E(best) < Ex) {
        sel = best;
      } else {
        const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
        const uint4 w = philox4x32_10(make_uint4(0u, (uint32_t)P.it, (uint32_t)q, 0x40000000u), key);
        const double u = u53(w.x, w.y);
        int Jmax = sed_J(E(0));
        for (int j = 1; j < m; ++j) Jmax = max(Jmax, sed_J(E(j)));
        double tot = 0.0;
        for (int j = 0; j < m; ++j) tot = __dadd_rn(tot, exp((double)(sed_J(E(j)) - Jmax)));
        const double target = __dmul_rn(u, tot);
        double run = 0.0;
        sel = m - 1;
        for (int j = 0; j < m; ++j) {
          run = __dadd_rn(run, exp((double)(sed_J(E(j)) - Jmax)));
          if (target < run) { sel = j; break; }
        }
      }
    }
    const double Es = E(sel);
    const int better = start || Es < P.Eb[q];
    P.sel[q] = sel;
    P.Ex[q] = Es;
    if (better) P.Eb[q] = Es;
    if (!start) P.iters[q] += 1;
    const int done = P.Eb[q] <= P.e_feas;
    P.done[q] = done;
    if (!done) atomicAdd(P.left, 1);
    s_sel = sel;
    s_better = better;
  }
  __syncthreads();
  const int n = P.n[q];
  const int64_t co = P.cdesc[(int64_t)q * P.M + s_sel].off;
  double2 *x = P.x + P.off[q], *xb = P.xb + P.off[q];
  const int better = s_better;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double2 v;
    if (P.from32) { const float2 f = P.c32[co + i]; v = make_double2(f.x, f.y); }
    else v = P.c64[co + i];
    x[i] = v;
    if (better) xb[i] = v;
  }
}

__global__ void sed_status_kernel(SedParams P, int32_t *status) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < P.num) status[q] = P.Eb[q] <= P.e_feas ? 0 : 3;
}

// The framework of Sec. 5.1: the search radius min(R_b, R*) of every instance.
__global__ void frame_radius_kernel(int num, const double *Rb, const double *Rbest, double *R) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < num) R[q] = fmin(Rb[q], Rbest[q]);
}

// The framework's record: instance q keeps (x, R) when R < R*.  One block per instance.
__global__ void frame_record_kernel(const int32_t *n, const int64_t *off, const double *Rn, const double2 *x,
                                    double *Rbest, double2 *xbest) {
  const int q = blockIdx.x;
  __shared__ int better;
  if (threadIdx.x == 0) {
    better = Rn[q] < Rbest[q];
    if (better) Rbest[q] = Rn[q];
  }
  __syncthreads();
  if (!better) return;
  const int64_t o = off[q];
  for (int i = threadIdx.x; i < n[q]; i += blockDim.x) xbest[o + i] = x[o + i];
}

__global__ void add_i32_kernel(int count, const int32_t *a, int32_t *acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) acc[i] += a[i];
}

}  // namespace

cudaError_t launch_add_i32(int count, const int32_t *a, int32_t *acc, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  add_i32_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, a, acc);
  return cudaGetLastError();
}

cudaError_t launch_frame_radius(int num, const double *Rb, const double *Rbest, double *R, cudaStream_t s) {
  if (num <= 0) return cudaSuccess;
  frame_radius_kernel<<<(num + 255) / 256, 256, 0, s>>>(num, Rb, Rbest, R);
  return cudaGetLastError();
}

cudaError_t launch_frame_record(const SedParams &p, const double *Rn, const double2 *x, double *Rbest,
                                double2 *xbest, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  frame_record_kernel<<<p.num, kSedT, 0, s>>>(p.n, p.off, Rn, x, Rbest, xbest);
  return cudaGetLastError();
}

cudaError_t launch_sed_status(const SedParams &p, int32_t *status, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  sed_status_kernel<<<(p.num + 255) / 256, 256, 0, s>>>(p, status);
  return cudaGetLastError();
}

cudaError_t launch_sed_init(const SedParams &p, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  sed_init_kernel<<<p.num, kSedT, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sed_prepare(const SedParams &p, int start, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  sed_prepare_kernel<<<p.num, kSedT, 0, s>>>(p, start);
  if (cudaError_t e = cudaGetLastError()) return e;
  sed_list_kernel<<<1, 1024, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sed_select(const SedParams &p, const double *Ecand, int start, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  sed_select_kernel<<<p.num, kSedT, 0, s>>>(p, Ecand, start);
  return cudaGetLastError();
}

}  // namespace pecc
