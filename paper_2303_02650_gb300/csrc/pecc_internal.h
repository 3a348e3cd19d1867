// pecc_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_bf16.h>

#include "pecc.h"
#include "pecc_dev.cuh"

namespace pecc {

// Cells per side the grid of an instance of n circles has at most: max(16, ceil(2 sqrt(n))).
__host__ __device__ inline int cell_grid_cap(int n) {
  const int cap = (int)ceil(2.0 * sqrt((double)n));
  return cap < 16 ? 16 : cap;
}

// Cell grid of one instance (the same arithmetic on the host and on the device, every operation
// correctly rounded): side l_cut (1 + margin), ncx = ceil(2R / side), capped at cell_grid_cap(n)
// cells per side (the side then grows to 2R / ncx).
__host__ __device__ inline void host_cell_grid(double R, double l_cut, int n, double *inv, int *nc,
                                               double margin = 1.0 / 1048576.0) {
  double cs = l_cut * (1.0 + margin);
  double iv = 1.0 / cs;
  double w = ceil((2.0 * R) * iv);
  const int cap = cell_grid_cap(n);
  int c = (w >= 1.0) ? (int)(w > 65535.0 ? 65535.0 : w) : 1;
  if (c > cap) {
    c = cap;
    iv = (double)c / (2.0 * R);
  }
  *inv = iv;
  *nc = c;
}

// The binary32 grid of the FP32 descent for an instance whose binary64 grid has ncx cells per side:
// side l_cut (1 + 2^-10), its inverse rounded down to binary32 (so the side only grows), at most
// ncx cells per side.
__host__ __device__ inline void f32_cell_grid(double R, double l_cut, int n, int ncx, float *inv_f, int *ncx_f) {
  double invf;
  int ncf;
  host_cell_grid(R, l_cut, n, &invf, &ncf, 1.0 / 1024.0);
  float f = (float)invf;
  if ((double)f > invf) f = nextafterf(f, 0.0f);
  *inv_f = f;
  *ncx_f = ncf < ncx ? ncf : ncx;
}

// Shared-memory share of a descent's outer neighbor list (list_outer > 0), in entries per circle;
// an outer list that outgrows it lives in global memory.
constexpr int kOuterPerCircle = 12;

// Message of the last failed call that has no context (read by pecc_last_error(NULL)).
void set_global_error(const char *msg);

// Everything a descent kernel reads or writes; device pointers into the context's buffers.
struct DescendParams {
  const InstDesc *desc;
  InstOut *out;
  int num;
  const int32_t *num_dev;  // if set: the instance count, read from device memory at launch (<= num)
  const int32_t *order;  // processing order of instances (largest first)
  int32_t *queue;        // work counter, zeroed before each launch
  float2 *x32;
  double2 *x64;
  void *xw, *xb, *xo;    // per-circle positions scratch (sized for double2)
  void *g, *gt, *d;      // per-circle vectors (sized for double2)
  void *S, *Y;           // (m + 1) secant slots per circle
  int32_t *perm;
  uint64_t *skey;
  int32_t *rp, *col;
  uint32_t *ckey;
  int32_t *corder, *cells;
  void *gram;
  int32_t *meta;
  double l_cut, rebuild_disp, step_max, e_tol, gsum_tol, c1, curv_eps, polish_gate;
  int m, max_iter, max_trials, anm, partition;
  uint64_t part_seed;     // random partition (3): Philox key
  double list_outer;     // > 0: reach of the outer list beyond l_cut (two-level lists)
  double stall_rel;       // FP32 phase: stop when E fell by less than this over stall_window sweeps
  int stall_window;
  const long long *t0;    // %globaltimer at the start of the call (written by stamp_kernel)
  long long budget_ns;    // 0 = no time budget
  int k_override;         // > 0: batches per instance for this phase (capped at the instance's k)
  size_t smem_bytes;      // dynamic shared memory per block for the working set
  // parity hook (pecc_set_list_dump): the lists in force at the end of each instance's phase and
  // the coordinates of their build; dump_cnt == nullptr: off
  int32_t *dump_cnt, *dump_col;
  double2 *dump_xb;
  int dump_stride;
};

cudaError_t launch_stamp(long long *t0, cudaStream_t s);

// Whole-GPU descent of one large instance (pecc_grid.cu).
struct GridCtl {
  unsigned int count, gen;  // barrier arrivals, generation
  int err, pad;             // a wait timed out
};
struct GridBufs {
  double *part;             // [grid][72] block partials
  double *res;              // [72] totals
  int32_t *ipart;           // [grid] block totals of integer scans
  int32_t *bucket;          // [2 (n / 4) + 2] partition buckets
  unsigned long long *hash; // [1] pair-set digest
  void *gram;               // [grid][kmax][kBasis^2] per-block Gram copies
  int kmax;
};
constexpr int kGridMinN = 16384;  // instances this large descend on the whole GPU
cudaError_t grid_descend_occupancy(int arith, int block, int *blocks_per_sm);
// Bounded-wait self-test of the grid barrier (synchronous, default stream).
cudaError_t selftest_grid_barrier(long long timeout_ns, int *failed_host, long long *waited_host);
cudaError_t launch_grid_descend(int arith, const DescendParams &p, int q, const GridBufs &g, GridCtl *c, int grid,
                                int block, cudaStream_t s);

// Launchers (pecc_descend.cu).  arith: PECC_FP64 (plain), PECC_FP32 (bulk), PECC_FP32_POLISH64 (polish).
// A compiled instance of the descent kernel: entry, launch bound (threads per block at most, and
// the resident blocks per SM its register budget is sized for), static shared memory.
struct DescendVariant {
  const void *fn;
  int max_threads, min_blocks;
  size_t static_smem;
};
int descend_variants(int arith, const DescendVariant **v);  // largest register budget first
int descend_variants32(const DescendVariant **v);
int descend_variants_fused(const DescendVariant **v);  // arith 3: FP32 descent + polish in one block
// the compiled instances of the fused kernel, one translation unit each (they compile in parallel)
DescendVariant descend_fused_256x2();
DescendVariant descend_fused_128x5();
DescendVariant descend_fused_512x1();
cudaError_t launch_descend_fused(const DescendVariant &v, const DescendParams &p32, const DescendParams &p64, int grid,
                                 int block, cudaStream_t s);
cudaError_t launch_descend(const DescendVariant &v, const DescendParams &p, int grid, int block, cudaStream_t s);
int descend_max_block(int arith);
size_t descend_smem_need(int arith, int n, int k, int ncx, int block, int m, bool outer);
size_t descend_smem_mandatory(int arith, int k, int block);

// Standalone kernels (pecc_kernels.cu).
// Container adjustment (pecc_adjust.cu).  Per-circle double2 arrays are the context's scratch
// (offset by the instance); S, Y: adjust_max_m() slots of double2 per circle.
struct AdjustParams {
  const InstDesc *desc;
  int num, from32;
  float2 *x32;
  double2 *x64;
  double *R;  // in/out, per instance
  double2 *g, *gn, *d, *zo, *xb, *xs, *sv, *S, *Y;
  int32_t *rp, *col;
  uint32_t *ckey;
  int32_t *corder, *cells;
  int32_t *iters, *status, *queue;
  int32_t *stats;  // optional: per instance {line-search trials, two-loop pair visits}
  double l_cut, rebuild_disp, step_max, gsum_tol, c1, curv_eps, lambda0;
  int m, max_iter, max_trials, anm, rounds;
};
// mixed != 0: the polish arithmetic for the pair terms (binary32 depths and forces) and binary32
// quasi-Newton vectors; energies, gradient storage and the radius stay binary64
cudaError_t launch_adjust(const AdjustParams &p, int mixed, int grid, cudaStream_t s);

// GBO with the explicit inverse Hessian per batch (pecc_dense.cu); binary64, per-circle scratch of
// the context (double2 each), H of instance q at H + h_off[q].
struct DenseParams {
  const InstDesc *desc;
  InstOut *out;
  int num;
  const int32_t *order;
  int32_t *queue;
  double2 *x, *g, *gn, *d, *xo, *xb, *xs, *hy;
  uint64_t *skey;
  int32_t *perm, *batch_of, *rp, *col;
  uint32_t *ckey;
  int32_t *corder, *cells;
  double *H;
  const int64_t *h_off;
  double l_cut, rebuild_disp, step_max, e_tol, gsum_tol, c1, curv_eps;
  int max_iter, max_trials, anm, partition;
  uint64_t part_seed;
};
cudaError_t launch_dense(const DenseParams &p, int grid, cudaStream_t s);
int64_t dense_h_words(int n, int k);

// SED over a batch (pecc_sed.cu).  Instance q: n[q] circles at off[q] of the operated (x) and best
// (xb) layouts; candidate slot q*M + j of the descent context (cdesc, cout, c64, c32).
struct SedParams {
  int num, M, it, init_mode, shared_r, from32;
  uint64_t seed;
  double amp, e_feas;
  const int32_t *n;
  const int64_t *off;
  const double *R;
  double2 *x, *xb;
  double *Ex, *Eb;
  int32_t *m, *sel, *done, *iters, *porder, *scan, *list;
  int32_t *count;   // active slots of this iteration (the descent's instance count)
  int32_t *active;  // instances with candidates this iteration
  int32_t *left;    // instances not done after this iteration's select
  const InstDesc *cdesc;
  const InstOut *cout;
  double2 *c64;
  float2 *c32;
};
cudaError_t launch_sed_init(const SedParams &p, cudaStream_t s);
cudaError_t launch_sed_prepare(const SedParams &p, int start, cudaStream_t s);  // prepare + active list
cudaError_t launch_sed_select(const SedParams &p, const double *Ecand, int start, cudaStream_t s);
cudaError_t launch_sed_status(const SedParams &p, int32_t *status, cudaStream_t s);
// The framework of Sec. 5.1 (pecc_sed.cu): R = min(R_b, R*); keep (x, R) where R < R*.
cudaError_t launch_frame_radius(int num, const double *Rb, const double *Rbest, double *R, cudaStream_t s);
cudaError_t launch_add_i32(int count, const int32_t *a, int32_t *acc, cudaStream_t s);  // acc += a
cudaError_t launch_frame_record(const SedParams &p, const double *Rn, const double2 *x, double *Rbest,
                                double2 *xbest, cudaStream_t s);
int adjust_max_m();

// Largest instance whose coordinates the block energy + gradient kernel stages in shared memory.
inline int energy_stage_n(int eval) { return (int)(PECC_ENERGY_STAGE_BYTES / (eval == 1 ? 8 : 16)); }

struct StandaloneParams {
  const InstDesc *desc;
  InstOut *out;
  int num;
  int64_t total;
  const int32_t *inst_of;
  float2 *x32;
  double2 *x64;
  void *xbuild;  // positions at the last standalone build (double2 size)
  int32_t *rp, *col;          // the standalone lists (one buffer per instance)
  uint32_t *ckey;
  int32_t *corder, *cells;
  int32_t *rp_t, *col_t;      // scratch lists of the feasibility check (the descent's buffers)
  uint32_t *ckey_t;
  int32_t *corder_t;
  void *xtmp;                 // per-circle double2 scratch
  void *xtmp2;                // another per-circle double2 scratch
  double l_cut, rebuild_disp;
  const int32_t *eorder;      // instances, largest first: block b of a per-instance kernel takes eorder[b]
};

cudaError_t launch_init(const StandaloneParams &p, uint64_t seed, int mode, int prec, cudaStream_t s);
cudaError_t launch_set_positions(const StandaloneParams &p, const double *xy, int prec, cudaStream_t s);
cudaError_t launch_get_positions(const StandaloneParams &p, double *xy, int from32, cudaStream_t s);
// Radii and cell grids of every instance from device radii (stream-ordered); a radius that is not
// finite and > 0 leaves R = NaN and a one-cell grid.
cudaError_t launch_set_radius(InstDesc *desc, const double *R, int num, double l_cut, cudaStream_t s);
cudaError_t launch_build(const StandaloneParams &p, int prec, int force, int32_t *rebuilt, int32_t *status,
                         int block, cudaStream_t s);
cudaError_t launch_energy_grad(const StandaloneParams &p, int eval, double *E, void *grad, void *ecirc,
                               int max_small_n, bool any_large, cudaStream_t s);
cudaError_t launch_feasible(const StandaloneParams &p, int from32, double tol, uint8_t *feasible,
                            double *max_overlap, int block, cudaStream_t s);
cudaError_t launch_export_csr(const StandaloneParams &p, const int64_t *base, int32_t *row_ptr, int32_t *col,
                              cudaStream_t s);
cudaError_t launch_export_cells(const StandaloneParams &p, uint32_t *key, int32_t *order, cudaStream_t s);
cudaError_t launch_nnz(const StandaloneParams &p, int64_t *nnz, cudaStream_t s);
cudaError_t launch_stats(const InstOut *out, int num, int32_t *stats, cudaStream_t s);
cudaError_t launch_outputs(const InstOut *out, int num, int32_t *iters, int32_t *status, double *E,
                           int32_t *builds, int32_t *changes, int32_t *trials, cudaStream_t s);

// Learned warm start (pecc_mlp.cu).
int mlp_num_params();
int mlp_num_bf16();
int mlp_train_blocks(int sms);
cudaError_t mlp_init(float *params, __nv_bfloat16 *wb, uint64_t seed, cudaStream_t s);
cudaError_t mlp_sync_bf16(const float *params, __nv_bfloat16 *wb, cudaStream_t s);
cudaError_t mlp_features(const StandaloneParams &p, float *feat, cudaStream_t s);
cudaError_t mlp_targets(const StandaloneParams &p, const double *xbefore, float *target, cudaStream_t s);
cudaError_t mlp_forward(const __nv_bfloat16 *wb, const float *params, const float *feat, int64_t rows, float *out,
                        int sms, cudaStream_t s, float *trace = nullptr);
cudaError_t mlp_grad(const __nv_bfloat16 *wb, const float *params, const float *feat, const float *target,
                     int64_t rows, float *part, float *lpart, float *grad, float *loss, int sms, cudaStream_t s,
                     float *fwd_trace = nullptr, float *bwd_trace = nullptr);
cudaError_t mlp_adam(float *params, float *m, float *v, const float *grad, __nv_bfloat16 *wb, float lr, int step,
                     cudaStream_t s);
cudaError_t mlp_apply(const StandaloneParams &p, const float *dout, float2 *backup, float max_move, cudaStream_t s);
cudaError_t mlp_revert(const StandaloneParams &p, const float2 *backup, const double *Eb, const double *Ea,
                       int32_t *accepted, cudaStream_t s);

}  // namespace pecc
