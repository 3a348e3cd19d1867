// pecc_kernels.cu -- standalone kernels: random init (Sec. 5.1), neighbor build
// (Sec. 4.3), fused energy + gradient (Eq. 3, Eq. 5), feasibility (Eq. 1, Eq. 2).
#include "pecc_internal.h"

namespace pecc {

namespace {

// Asynchronous copy of BYTES (8 or 16) from global to shared memory (cp.async; completed by
// cp.async.wait_all).  Both addresses must be BYTES-aligned.
template <int BYTES> __device__ __forceinline__ void cp_async_shared(void *dst, const void *src) {
  static_assert(BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}

// threads per block of the block-per-instance energy + gradient kernel (measured on the
// 4096-instance batch's final layouts: 128 threads 41.2 us, 256 threads 43.3 us, 512 threads 49.5 us)
constexpr int kEgBlock = 128;

// ------------------------------------------------------------------ init ----
// Circle i of instance q: Philox4x32-10, key (seed lo, seed hi), counter (i, attempt, q, 0);
// (w0, w1) and (w2, w3) give two 53-bit uniforms u, v; candidate (R-1)(2u-1, 2v-1),
// accepted inside the disk of radius R-1 (mode 0), or R (2u-1, 2v-1) in the square (mode 1).
__global__ void init_kernel(StandaloneParams P, uint64_t seed, int mode, int prec) {
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const int q = P.inst_of[gi];
  const InstDesc D = P.desc[q];
  const uint32_t i = (uint32_t)(gi - D.off);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const double R = D.R, rr = __dsub_rn(R, 1.0);
  double x = 0.0, y = 0.0;
  if (mode == 1) {
    uint4 w = philox4x32_10(make_uint4(i, 0u, (uint32_t)q, 0u), key);
    x = __dmul_rn(R, __dsub_rn(__dmul_rn(2.0, u53(w.x, w.y)), 1.0));
    y = __dmul_rn(R, __dsub_rn(__dmul_rn(2.0, u53(w.z, w.w)), 1.0));
  } else if (rr > 0.0) {
    for (uint32_t a = 0; a < 64u; ++a) {
      uint4 w = philox4x32_10(make_uint4(i, a, (uint32_t)q, 0u), key);
      double cx = __dmul_rn(rr, __dsub_rn(__dmul_rn(2.0, u53(w.x, w.y)), 1.0));
      double cy = __dmul_rn(rr, __dsub_rn(__dmul_rn(2.0, u53(w.z, w.w)), 1.0));
      if (__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)) <= __dmul_rn(rr, rr)) { x = cx; y = cy; break; }
    }
  }
  if (prec == 0) {
    P.x64[gi] = make_double2(x, y);
  } else {
    float2 f = make_float2((float)x, (float)y);
    P.x32[gi] = f;
    P.x64[gi] = make_double2((double)f.x, (double)f.y);
  }
}

__global__ void set_pos_kernel(StandaloneParams P, const double *__restrict__ xy, int prec) {
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  double x = xy[2 * gi], y = xy[2 * gi + 1];
  if (prec == 0) {
    P.x64[gi] = make_double2(x, y);
  } else {
    float2 f = make_float2((float)x, (float)y);
    P.x32[gi] = f;
    P.x64[gi] = make_double2((double)f.x, (double)f.y);
  }
}

__global__ void get_pos_kernel(StandaloneParams P, double *__restrict__ xy, int from32) {
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  double2 v;
  if (from32) { float2 f = P.x32[gi]; v = make_double2((double)f.x, (double)f.y); }
  else v = P.x64[gi];
  xy[2 * gi] = v.x;
  xy[2 * gi + 1] = v.y;
}

__global__ void set_radius_kernel(InstDesc *desc, const double *__restrict__ R, int num, double l_cut) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= num) return;
  InstDesc &D = desc[q];
  const double r = R[q];
  double inv;
  int nc;
  float invf;
  int ncf;
  if (r > 0.0 && isfinite(r)) {
    host_cell_grid(r, l_cut, D.n, &inv, &nc);
    f32_cell_grid(r, l_cut, D.n, nc, &invf, &ncf);
    D.R = r;
  } else {  // the instance's energies, descents and checks come out NaN (status PECC_DESC_NONFINITE)
    host_cell_grid(1.0, l_cut, D.n, &inv, &nc);
    f32_cell_grid(1.0, l_cut, D.n, nc, &invf, &ncf);
    nc = ncf = 1;
    D.R = __longlong_as_double(0x7ff8000000000000ll);
  }
  D.inv_cs = inv;
  D.ncx = nc;
  D.inv_f = invf;
  D.ncx_f = ncf;
}

// ----------------------------------------------------------------- build ----
template <typename T>
__global__ void build_kernel(StandaloneParams P, int force, int32_t *rebuilt, int32_t *status) {
  __shared__ int32_t sh[40];
  using PP = v2<T>;
  const int q = blockIdx.x;
  const InstDesc D = P.desc[q];
  const int n = D.n;
  const PP *x;
  if constexpr (sizeof(T) == 4) x = (const PP *)(P.x32 + D.off);
  else x = (const PP *)(P.x64 + D.off);
  PP *xb = (PP *)P.xbuild + D.off;
  int go = force;
  if (!go) {
    // largest displacement since the last standalone build
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      PP a = x[i], b = xb[i];
      double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y;
      m = fmax(m, dx * dx + dy * dy);
    }
    go = __syncthreads_or(m > P.rebuild_disp * P.rebuild_disp);
  }
  if (go) {
    const T lc2 = (T)(P.l_cut * P.l_cut);
    CellGrid G{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
    int tot = cta_build_neighbors<T, int32_t>(x, n, G, lc2, P.ckey + D.off, P.corder + D.off, P.cells + D.cell_off,
                                     (PP *)P.xtmp + D.off, P.rp + D.off + q, P.col + D.col_s_off, D.cap, sh,
                                     nullptr, true);
    for (int i = threadIdx.x; i < n; i += blockDim.x) xb[i] = x[i];
    if (threadIdx.x == 0 && status) status[q] = tot > D.cap ? 4 : 0;
  } else if (threadIdx.x == 0 && status) {
    status[q] = 0;
  }
  if (threadIdx.x == 0 && rebuilt) rebuilt[q] = go;
}

// ------------------------------------------------- fused energy + gradient ----
// One thread per circle (gather over its row, no atomics):
//   g_i = sum_{j in Gamma(i)} -2 d_ij (c_i - c_j) / l_ij + 2 d_i0 c_i / |c_i|
//   e_i = sum_{j in Gamma(i), j < i} d_ij^2 + d_i0^2      (so that E = sum_i e_i, Eq. 5)
template <class A>
__global__ void __launch_bounds__(256) energy_grad_kernel(StandaloneParams P, int stage_n, void *__restrict__ grad_,
                                                          void *__restrict__ ecirc_) {
  using pos_t = typename A::pos_t;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  using PP = v2<pos_t>;
  using VV = v2<vec_t>;
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  const int q = __ldg(P.inst_of + gi);
  if (P.desc[q].n <= stage_n) return;  // the block kernel's instance
  const int64_t off = P.desc[q].off;
  const int64_t col_off = P.desc[q].col_s_off;
  const double Rd = P.desc[q].R;
  const acc_t R = (acc_t)Rd;
  const acc_t Rm1sq = (acc_t)((Rd >= 1.0) ? (Rd - 1.0) * (Rd - 1.0) : -1.0);
  const PP *x = (sizeof(pos_t) == 4) ? (const PP *)(P.x32 + off) : (const PP *)(P.x64 + off);
  const int i = (int)(gi - off);
  const int32_t *rp = P.rp + off + q;
  const int32_t *cl = P.col + col_off;
  PP xi = x[i];
  vec_t gx = 0, gy = 0;
  acc_t e = 0;
  const int lo = __ldg(rp + i), hi = __ldg(rp + i + 1);
  if (__ldg(rp + P.desc[q].n) > P.desc[q].cap) {  // the last build overflowed the list's capacity: no valid list
    VV gv; gv.x = gv.y = (vec_t)NAN;
    ((VV *)grad_)[gi] = gv;
    ((acc_t *)ecirc_)[gi] = (acc_t)NAN;
    return;
  }
  // two entries per step (their index and coordinate loads in flight together); the sums take the
  // entries in row order
  for (int t = lo; t < hi; t += 2) {
    const bool two = t + 1 < hi;
    const int j1 = __ldg(cl + t);
    const int j2 = two ? __ldg(cl + t + 1) : j1;
    const PP x1 = x[j1], x2 = x[j2];
    vec_t fx, fy;
    const acc_t d1 = A::pair(xi, x1, fx, fy);
    gx += fx; gy += fy;
    if (j1 < i) e += d1 * d1;
    if (two) {
      const acc_t d2 = A::pair(xi, x2, fx, fy);
      gx += fx; gy += fy;
      if (j2 < i) e += d2 * d2;
    }
  }
  vec_t fx, fy;
  acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
  gx += fx; gy += fy;
  e += d0 * d0;
  VV gv; gv.x = gx; gv.y = gy;
  ((VV *)grad_)[gi] = gv;
  ((acc_t *)ecirc_)[gi] = e;
}

// One block per instance whose coordinates fit the staging limit (stage_n circles at most): the
// coordinates are staged in shared memory by one coalesced read, so every neighbor gather is an
// on-chip load; row pointers and lists stream through once, the gradient is written once, and the
// energy is reduced in the block in a fixed order (deterministic) and written once.  Larger
// instances are left to energy_grad_kernel + energy_reduce_kernel.  Blocks take the instances
// largest first (the last blocks to start are the shortest), kEgBlock threads each: sixteen
// blocks share an SM.
template <class A>
__global__ void __launch_bounds__(kEgBlock) energy_grad_block_kernel(StandaloneParams P, int stage_n,
                                                                void *__restrict__ grad_, double *E) {
  using pos_t = typename A::pos_t;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  using PP = v2<pos_t>;
  using VV = v2<vec_t>;
  extern __shared__ __align__(16) unsigned char stage[];
  __shared__ acc_t red[32];
  const int q = P.eorder[blockIdx.x];
  const int n = P.desc[q].n;
  if (n > stage_n) return;  // the per-circle kernels' instance (uniform across the block)
  if (n == 0) {
    if (threadIdx.x == 0) E[q] = 0.0;
    return;
  }
  const int64_t off = P.desc[q].off;
  const int64_t col_off = P.desc[q].col_s_off;
  const double Rd = P.desc[q].R;
  const acc_t R = (acc_t)Rd;
  const acc_t Rm1sq = (acc_t)((Rd >= 1.0) ? (Rd - 1.0) * (Rd - 1.0) : -1.0);
  const PP *x = (sizeof(pos_t) == 4) ? (const PP *)(P.x32 + off) : (const PP *)(P.x64 + off);
  const int32_t *rp = P.rp + off + q;
  const int32_t *cl = P.col + col_off;
  VV *grad = (VV *)grad_ + off;
  const int end = __ldg(rp + n);  // in flight with the coordinates
  PP *xs = (PP *)stage;
  // the staging copies are asynchronous (cp.async, 8 or 16 bytes each): all of a thread's copies
  // are in flight together instead of one load round trip per coordinate
  for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async_shared<sizeof(PP)>(xs + i, x + i);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (end > P.desc[q].cap) {  // the last build overflowed the list's capacity: no valid list
    for (int i = threadIdx.x; i < n; i += blockDim.x) { VV gv; gv.x = gv.y = (vec_t)NAN; grad[i] = gv; }
    if (threadIdx.x == 0) E[q] = NAN;
    return;
  }
  __syncthreads();
  acc_t e = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const PP xi = xs[i];
    vec_t gx = 0, gy = 0;
    const int lo = __ldg(rp + i), hi = __ldg(rp + i + 1);
    // two entries per step (both loads in flight); the sums take the entries in row order
    for (int t = lo; t < hi; t += 2) {
      const bool two = t + 1 < hi;
      const int j1 = __ldg(cl + t);
      const int j2 = two ? __ldg(cl + t + 1) : j1;
      const PP x1 = xs[j1], x2 = xs[j2];
      vec_t fx, fy;
      const acc_t d1 = A::pair_skip(xi, x1, fx, fy);
      gx += fx; gy += fy;
      if (j1 < i) e += d1 * d1;
      if (two) {
        const acc_t d2 = A::pair_skip(xi, x2, fx, fy);
        gx += fx; gy += fy;
        if (j2 < i) e += d2 * d2;
      }
    }
    vec_t fx, fy;
    acc_t d0 = A::wall(xi, R, Rm1sq, fx, fy);
    gx += fx; gy += fy;
    e += d0 * d0;
    VV gv; gv.x = gx; gv.y = gy;
    grad[i] = gv;
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc_t v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : acc_t(0);
    v = warp_sum(v);
    if (threadIdx.x == 0) E[q] = (double)v;
  }
}

// Per-instance sum of the per-circle energies (fixed order: deterministic), for the instances the
// block kernel left (more than stage_n circles).  Each thread keeps kRed partial sums over
// interleaved circles, so that kRed loads are in flight at a time, and adds them in a fixed order.
constexpr int kRed = 8;
template <typename acc_t>
__global__ void __launch_bounds__(1024) energy_reduce_kernel(StandaloneParams P, int stage_n,
                                                             const acc_t *__restrict__ ecirc, double *E) {
  __shared__ acc_t sh[32];
  const int q = blockIdx.x;
  const InstDesc D = P.desc[q];
  if (D.n <= stage_n) return;
  const acc_t *e = ecirc + D.off;
  const int B = blockDim.x;
  acc_t part[kRed];
#pragma unroll
  for (int u = 0; u < kRed; ++u) part[u] = 0;
  for (int i0 = threadIdx.x; i0 < D.n; i0 += kRed * B) {
#pragma unroll
    for (int u = 0; u < kRed; ++u) {
      const int i = i0 + u * B;
      if (i < D.n) part[u] += e[i];
    }
  }
  acc_t s = part[0];
#pragma unroll
  for (int u = 1; u < kRed; ++u) s += part[u];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc_t v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : acc_t(0);
    v = warp_sum(v);
    if (threadIdx.x == 0) E[q] = (double)v;
  }
}

// ----------------------------------------------------------- feasibility ----
// A fresh FP64 list with cutoff l_cut > 2 holds every pair with l_ij < 2, so the largest
// depth over the list equals the largest over all pairs (Eq. 1); walls per circle (Eq. 2).
__global__ void feasible_kernel(StandaloneParams P, int from32, double tol, uint8_t *feasible,
                                double *max_overlap) {
  __shared__ int32_t sh[40];
  __shared__ double red[32];
  const int q = P.eorder[blockIdx.x];  // largest instance first
  const InstDesc D = P.desc[q];
  const int n = D.n;
  double2 *x = (double2 *)P.xtmp + D.off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (from32) { float2 f = P.x32[D.off + i]; x[i] = make_double2((double)f.x, (double)f.y); }
    else x[i] = P.x64[D.off + i];
  }
  __syncthreads();
  int32_t *rp = P.rp_t + D.rp_off;
  int32_t *cl = P.col_t + D.col_off;
  const double lc2 = P.l_cut * P.l_cut;
  CellGrid G{D.R, D.inv_cs, 0.f, 0.f, D.ncx, false};
  int tot = cta_build_neighbors<double, int32_t>(x, n, G, lc2, P.ckey_t + D.off, P.corder_t + D.off, P.cells + D.cell_off,
                                        (double2 *)P.xtmp2 + D.off, rp, cl, 2 * D.cap, sh, nullptr, false);
  double m = 0.0;
  int bad = 0;
  if (tot <= 2 * D.cap) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double2 xi = x[i];
      bad |= !(isfinite(xi.x) && isfinite(xi.y));
      for (int t = rp[i]; t < rp[i + 1]; ++t) {
        int j = cl[t];
        if (j > i) m = fmax(m, pair_depth_exact(xi, x[j]));
      }
      m = fmax(m, wall_depth_exact(xi, D.R));
    }
  } else {
    bad = 1;
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
    if (bad) v = __longlong_as_double(0x7ff8000000000000ll);  // NaN: not checkable
    bool ok = !bad && v <= tol;
    if (feasible) feasible[q] = ok ? 1 : 0;
    if (max_overlap) max_overlap[q] = v;
    P.out[q].max_overlap = v;
  }
}

// ---------------------------------------------------------------- export ----
__global__ void export_csr_kernel(StandaloneParams P, const int64_t *__restrict__ base, int32_t *row_ptr,
                                  int32_t *col) {
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) {
    if (gi == P.total && P.num > 0) row_ptr[P.total] = (int32_t)base[P.num];
    return;
  }
  const int q = P.inst_of[gi];
  const InstDesc D = P.desc[q];
  const int i = (int)(gi - D.off);
  const int32_t *rp = P.rp + D.off + q;
  const int lo = rp[i], hi = rp[i + 1];
  const int64_t b = base[q];
  row_ptr[gi] = (int32_t)(b + lo);
  for (int t = lo; t < hi; ++t) col[b + t] = (int32_t)(D.off + P.col[D.col_s_off + t]);
}

__global__ void export_cells_kernel(StandaloneParams P, uint32_t *key, int32_t *order) {
  int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P.total) return;
  key[gi] = P.ckey[gi];
  order[gi] = P.corder[gi];
}

__global__ void nnz_kernel(StandaloneParams P, int64_t *nnz) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.num) return;
  const InstDesc D = P.desc[q];
  nnz[q] = (int64_t)P.rp[D.off + q + D.n];
}

__global__ void outputs_kernel(const InstOut *out, int num, int32_t *iters, int32_t *status, double *E,
                               int32_t *builds, int32_t *changes, int32_t *trials) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= num) return;
  if (iters) iters[q] = out[q].iters;
  if (status) status[q] = out[q].status;
  if (E) E[q] = out[q].E;
  if (builds) builds[q] = out[q].builds;
  if (changes) changes[q] = out[q].changes;
  if (trials) trials[q] = out[q].trials;
}

__global__ void stats_kernel(const InstOut *out, int num, int32_t *st) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= num) return;
  const InstOut o = out[q];
  int32_t *r = st + 10 * (int64_t)q;
  r[0] = o.iters; r[1] = o.status; r[2] = o.builds; r[3] = o.changes; r[4] = o.trials;
  r[5] = o.resets; r[6] = o.stalls; r[7] = o.polished; r[8] = o.iters32; r[9] = o.trials32;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_init(const StandaloneParams &p, uint64_t seed, int mode, int prec, cudaStream_t s) {
  if (p.total > 0) init_kernel<<<blocks_for(p.total, 256), 256, 0, s>>>(p, seed, mode, prec);
  return cudaGetLastError();
}

cudaError_t launch_set_positions(const StandaloneParams &p, const double *xy, int prec, cudaStream_t s) {
  if (p.total > 0) set_pos_kernel<<<blocks_for(p.total, 256), 256, 0, s>>>(p, xy, prec);
  return cudaGetLastError();
}

cudaError_t launch_get_positions(const StandaloneParams &p, double *xy, int from32, cudaStream_t s) {
  if (p.total > 0) get_pos_kernel<<<blocks_for(p.total, 256), 256, 0, s>>>(p, xy, from32);
  return cudaGetLastError();
}

cudaError_t launch_set_radius(InstDesc *desc, const double *R, int num, double l_cut, cudaStream_t s) {
  if (num > 0) set_radius_kernel<<<blocks_for(num, 128), 128, 0, s>>>(desc, R, num, l_cut);
  return cudaGetLastError();
}

cudaError_t launch_build(const StandaloneParams &p, int prec, int force, int32_t *rebuilt, int32_t *status,
                         int block, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  if (prec == 1) build_kernel<float><<<p.num, block, 0, s>>>(p, force, rebuilt, status);
  else build_kernel<double><<<p.num, block, 0, s>>>(p, force, rebuilt, status);
  return cudaGetLastError();
}

template <class A> static cudaError_t launch_eg_block(const StandaloneParams &p, int stage_n, size_t smem,
                                                     void *grad, double *E, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(energy_grad_block_kernel<A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  energy_grad_block_kernel<A><<<p.num, kEgBlock, smem, s>>>(p, stage_n, grad, E);
  return cudaGetLastError();
}

// max_small_n: the largest instance of at most stage_n(eval) circles (-1: none; instances of 0
// circles get E = 0 from the block kernel); any_large: some instance has more.
cudaError_t launch_energy_grad(const StandaloneParams &p, int eval, double *E, void *grad, void *ecirc,
                               int max_small_n, bool any_large, cudaStream_t s) {
  if (p.num <= 0) return cudaSuccess;
  const int stage_n = energy_stage_n(eval);
  cudaError_t e = cudaSuccess;
  if (max_small_n >= 0) {
    const size_t smem = std::max<size_t>(16, (size_t)max_small_n * (eval == 1 ? sizeof(float2) : sizeof(double2)));
    if (eval == 0) e = launch_eg_block<Arith64>(p, stage_n, smem, grad, E, s);
    else if (eval == 1) e = launch_eg_block<Arith32>(p, stage_n, smem, grad, E, s);
    else e = launch_eg_block<ArithMix>(p, stage_n, smem, grad, E, s);
    if (e != cudaSuccess) return e;
  }
  if (any_large && p.total > 0) {
    unsigned nb = blocks_for(p.total, 256);
    if (eval == 0) energy_grad_kernel<Arith64><<<nb, 256, 0, s>>>(p, stage_n, grad, ecirc);
    else if (eval == 1) energy_grad_kernel<Arith32><<<nb, 256, 0, s>>>(p, stage_n, grad, ecirc);
    else energy_grad_kernel<ArithMix><<<nb, 256, 0, s>>>(p, stage_n, grad, ecirc);
    if (eval == 1) energy_reduce_kernel<float><<<p.num, 1024, 0, s>>>(p, stage_n, (const float *)ecirc, E);
    else energy_reduce_kernel<double><<<p.num, 1024, 0, s>>>(p, stage_n, (const double *)ecirc, E);
  }
  return cudaGetLastError();
}

cudaError_t launch_feasible(const StandaloneParams &p, int from32, double tol, uint8_t *feasible,
                            double *max_overlap, int block, cudaStream_t s) {
  if (p.num > 0) feasible_kernel<<<p.num, block, 0, s>>>(p, from32, tol, feasible, max_overlap);
  return cudaGetLastError();
}

cudaError_t launch_export_csr(const StandaloneParams &p, const int64_t *base, int32_t *row_ptr, int32_t *col,
                              cudaStream_t s) {
  export_csr_kernel<<<blocks_for(p.total + 1, 256), 256, 0, s>>>(p, base, row_ptr, col);
  return cudaGetLastError();
}

cudaError_t launch_export_cells(const StandaloneParams &p, uint32_t *key, int32_t *order, cudaStream_t s) {
  if (p.total > 0) export_cells_kernel<<<blocks_for(p.total, 256), 256, 0, s>>>(p, key, order);
  return cudaGetLastError();
}

cudaError_t launch_nnz(const StandaloneParams &p, int64_t *nnz, cudaStream_t s) {
  if (p.num > 0) nnz_kernel<<<blocks_for(p.num, 128), 128, 0, s>>>(p, nnz);
  return cudaGetLastError();
}

cudaError_t launch_outputs(const InstOut *out, int num, int32_t *iters, int32_t *status, double *E,
                           int32_t *builds, int32_t *changes, int32_t *trials, cudaStream_t s) {
  if (num > 0) outputs_kernel<<<blocks_for(num, 128), 128, 0, s>>>(out, num, iters, status, E, builds, changes, trials);
  return cudaGetLastError();
}

cudaError_t launch_stats(const InstOut *out, int num, int32_t *stats, cudaStream_t s) {
  if (num > 0) stats_kernel<<<blocks_for(num, 128), 128, 0, s>>>(out, num, stats);
  return cudaGetLastError();
}

}  // namespace pecc
