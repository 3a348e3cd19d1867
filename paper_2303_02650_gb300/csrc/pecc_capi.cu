// pecc_capi.cu -- the C ABI (include/pecc.h): context, device buffers, launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pecc.h"
#include "pecc_internal.h"

using namespace pecc;

struct pecc_ctx {
  pecc_config cfg{};
  std::vector<int32_t> n;
  std::vector<int32_t> k;
  int num = 0;
  int64_t total = 0;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 1;
  std::vector<InstDesc> desc_h;
  std::vector<void *> allocs;
  // device buffers
  InstDesc *desc = nullptr;
  InstOut *out = nullptr;
  int32_t *order = nullptr, *queue = nullptr, *inst_of = nullptr;
  int32_t *eorder = nullptr;  // largest instance first, never rewritten (the standalone kernels' block order)
  long long *t0 = nullptr;
  float2 *x32 = nullptr;
  double2 *x64 = nullptr;
  void *xw = nullptr, *xb = nullptr, *xo = nullptr, *g = nullptr, *gt = nullptr, *d = nullptr, *xbuild = nullptr;
  void *S = nullptr, *Y = nullptr, *gram = nullptr, *ecirc = nullptr;
  int32_t *perm = nullptr, *meta = nullptr;
  uint64_t *skey = nullptr;
  int32_t *rp = nullptr, *col = nullptr, *rp_s = nullptr, *col_s = nullptr;
  double2 *adjS = nullptr, *adjY = nullptr;  // binary64 secant pairs of the container adjustment
  int32_t *num_dev = nullptr;  // set by an owning search (SED): the descent's instance count on the device
  double *denseH = nullptr;    // qn_dense: the inverse Hessians of every batch (allocated on first use)
  int64_t *dense_hoff = nullptr;
  bool dense_ran = false;
  uint32_t *ckey = nullptr, *ckey_s = nullptr;
  int32_t *corder = nullptr, *corder_s = nullptr, *cells = nullptr;
  int64_t *nnz = nullptr;
  char *stage = nullptr;  // per-instance staging of pecc_solve_host (R, outputs)
  bool radius_set = false;
  bool radius_host_known = false;  // radius_host holds the radii of the last pecc_solve_host
  std::vector<double> radius_host;
  int lists_prec = -1;  // precision of the standalone lists: 0 FP64, 1 FP32
  int block = 0, bps = 0, grid = 0, block_build = 256;
  // per arithmetic (0 FP64, 1 FP32, 2 polish) and 3 = FP32 descent + polish fused in one kernel
  struct Launch { int block = 0, bps = 0, grid = 0, var = 0; size_t smem = 0; } lc[4];
  bool lc_ready = false;
  bool tuned = false;  // launch shapes chosen by pecc_autotune
  int tuned_block = 0, tuned_bps = 0;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // whole-GPU descent of large instances
  std::vector<int> big;
  GridBufs gb{};
  GridCtl *gctl = nullptr;
  int ggrid = 0, gblock = 256;
  // learned warm start scratch (allocated on first use)
  float *feat = nullptr, *dout = nullptr;
  float2 *backup = nullptr;
  double *Eb = nullptr, *Ea = nullptr;
  // parity hook of pecc_set_list_dump (caller's device buffers; nullptr = off)
  int32_t *dump_cnt = nullptr, *dump_col = nullptr;
  double *dump_xb = nullptr;
  int dump_stride = 0;
  std::string err;
};

static std::string g_create_err;

namespace pecc {
void set_global_error(const char *msg) { g_create_err = msg; }
}  // namespace pecc

static pecc_status fail(pecc_ctx *c, pecc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_err = buf;
  return s;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(ctx, PECC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T> static pecc_status dalloc(pecc_ctx *ctx, T **p, size_t count) {
  void *v = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e != cudaSuccess) return fail(ctx, PECC_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  ctx->allocs.push_back(v);
  *p = (T *)v;
  return PECC_OK;
}

static StandaloneParams sparams(pecc_ctx *c) {
  StandaloneParams p{};
  p.desc = c->desc;
  p.out = c->out;
  p.num = c->num;
  p.total = c->total;
  p.inst_of = c->inst_of;
  p.x32 = c->x32;
  p.x64 = c->x64;
  p.xbuild = c->xbuild;
  p.rp = c->rp_s;
  p.col = c->col_s;
  p.ckey = c->ckey_s;
  p.corder = c->corder_s;
  p.cells = c->cells;
  p.rp_t = c->rp;
  p.col_t = c->col;
  p.ckey_t = c->ckey;
  p.corder_t = c->corder;
  p.xtmp = c->xw;
  p.xtmp2 = c->xo;
  p.l_cut = c->cfg.l_cut;
  p.rebuild_disp = c->cfg.rebuild_disp;
  p.eorder = c->eorder;
  return p;
}

extern "C" {

void pecc_config_default(pecc_config *c) {
  std::memset(c, 0, sizeof *c);
  c->precision = PECC_FP32_POLISH64;
  c->l_cut = 2.5;
  c->rebuild_disp = 0.25;
  c->step_max = 0.1;
  c->lbfgs_m = 10;
  c->max_iter = 2000;
  c->polish_max_iter = 1000;
  c->k_batches = 0;
  c->partition = PECC_PART_SECTOR;
  c->max_trials = 30;
  c->anm = 1;
  c->init_mode = PECC_INIT_DISK;
  c->e_tol = 1e-20;
  c->gsum_tol = 1e-12;
  c->c1 = 1e-4;
  c->curv_eps = 1e-10;
  c->polish_gate = 1e-4;
  c->feas_tol = 1e-9;
  c->nbr_capacity = 16.0;
  c->time_budget_ns = 0;
  c->block_threads = 0;
  c->blocks_per_sm = 0;
  c->stall_rel = 1e-3;
  c->stall_window = 10;
  c->polish_k = 1;
  c->polish_stall_rel = 1e-2;
  c->polish_stall_window = 100;
  c->fuse_phases = 1;
  c->list_outer = 0.5;
}

static int default_k(int n) { return n < 300 ? 1 : (n < 500 ? 3 : 5); }

pecc_status pecc_create(const pecc_config *cfg, void *stream, pecc_ctx **out) {
  if (!out) return fail(nullptr, PECC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, PECC_ERR_ARG, "cfg is NULL");
  if (cfg->num_instances < 0 || (cfg->num_instances > 0 && !cfg->n))
    return fail(nullptr, PECC_ERR_ARG, "num_instances < 0 or n is NULL");
  if (cfg->precision < 0 || cfg->precision > 2) return fail(nullptr, PECC_ERR_ARG, "bad precision");
  if (!(cfg->l_cut > 2.0)) return fail(nullptr, PECC_ERR_ARG, "l_cut must exceed 2");
  if (!(cfg->rebuild_disp > 0.0) || !(cfg->step_max > 0.0) || !(2.0 * cfg->rebuild_disp > cfg->step_max))
    return fail(nullptr, PECC_ERR_ARG, "need 0 < step_max < 2 * rebuild_disp");
  if (2.0 * cfg->rebuild_disp > cfg->l_cut - 2.0 + 1e-12)
    return fail(nullptr, PECC_ERR_ARG, "rebuild_disp must be <= (l_cut - 2) / 2");
  if (cfg->lbfgs_m < 1 || cfg->lbfgs_m > kMaxSlots - 1) return fail(nullptr, PECC_ERR_ARG, "lbfgs_m must be in 1..10");
  if (cfg->max_iter < 0 || cfg->polish_max_iter < 0 || cfg->max_trials < 1)
    return fail(nullptr, PECC_ERR_ARG, "bad iteration limits");
  if (cfg->k_batches < 0 || cfg->k_batches > kMaxK) return fail(nullptr, PECC_ERR_ARG, "k_batches must be in 0..64");
  if (cfg->partition < 0 || cfg->partition > 3) return fail(nullptr, PECC_ERR_ARG, "bad partition");
  if (cfg->init_mode < 0 || cfg->init_mode > 1) return fail(nullptr, PECC_ERR_ARG, "bad init_mode");
  if (!(cfg->nbr_capacity >= 1.0)) return fail(nullptr, PECC_ERR_ARG, "nbr_capacity must be >= 1");
  if (cfg->stall_window < 0 || !(cfg->stall_rel >= 0.0)) return fail(nullptr, PECC_ERR_ARG, "bad stall rule");
  if (cfg->polish_stall_window < 0 || !(cfg->polish_stall_rel >= 0.0))
    return fail(nullptr, PECC_ERR_ARG, "bad polish stall rule");
  if (cfg->polish_k < 0 || cfg->polish_k > kMaxK) return fail(nullptr, PECC_ERR_ARG, "polish_k must be in 0..64");
  if (cfg->smem_per_block < 0) return fail(nullptr, PECC_ERR_ARG, "smem_per_block must be >= 0");
  if (cfg->qn_dense != 0 && cfg->qn_dense != 1) return fail(nullptr, PECC_ERR_ARG, "qn_dense must be 0 or 1");
  if (!(cfg->list_outer == 0.0 || (cfg->list_outer >= 1.0 / 512.0 && cfg->list_outer <= 64.0)))
    return fail(nullptr, PECC_ERR_ARG, "list_outer must be 0 or in [2^-9, 64]");
  if (cfg->qn_dense && cfg->precision != PECC_FP64)
    return fail(nullptr, PECC_ERR_ARG, "qn_dense needs precision PECC_FP64");
  if (cfg->block_threads != 0 && (cfg->block_threads < 32 || cfg->block_threads % 32 ||
                                  cfg->block_threads > descend_max_block(cfg->precision == PECC_FP64 ? 0 : 1)))
    return fail(nullptr, PECC_ERR_ARG, "block_threads must be a multiple of 32 within the kernel's limit");
  if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32) return fail(nullptr, PECC_ERR_ARG, "blocks_per_sm must be in 0..32");
  int64_t total = 0;
  for (int q = 0; q < cfg->num_instances; ++q) {
    if (cfg->n[q] < 0) return fail(nullptr, PECC_ERR_ARG, "n[%d] < 0", q);
    total += cfg->n[q];
  }
  if (total > (int64_t)1 << 30) return fail(nullptr, PECC_ERR_ARG, "too many circles");

  pecc_ctx *ctx = new pecc_ctx();
  ctx->cfg = *cfg;
  ctx->cfg.n = nullptr;
  ctx->num = cfg->num_instances;
  ctx->n.assign(cfg->n, cfg->n + ctx->num);
  ctx->total = total;
  ctx->stream = (cudaStream_t)stream;
  auto bail = [&](pecc_status s) {
    g_create_err = ctx->err;
    pecc_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(fail(ctx, PECC_ERR_CUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);

  const int m1 = cfg->lbfgs_m + 1;
  const bool fp64 = cfg->precision == PECC_FP64;
  const size_t vec2 = fp64 ? sizeof(double2) : sizeof(float2);
  const size_t vecs = fp64 ? sizeof(double) : sizeof(float);
  ctx->desc_h.resize(ctx->num);
  ctx->k.resize(ctx->num);
  int64_t off = 0, rp_off = 0, col_off = 0, col_s_off = 0, gram_off = 0, meta_off = 0, cell_off = 0;
  for (int q = 0; q < ctx->num; ++q) {
    InstDesc &D = ctx->desc_h[q];
    std::memset(&D, 0, sizeof D);
    const int n = ctx->n[q];
    int k = cfg->k_batches > 0 ? cfg->k_batches : default_k(n);
    k = std::max(1, std::min(k, std::max(n, 1)));
    ctx->k[q] = k;
    D.n = n;
    D.k = k;
    D.big = n >= kGridMinN ? 1 : 0;
    if (D.big) ctx->big.push_back(q);
    D.cap = (int32_t)std::min<double>(std::ceil(cfg->nbr_capacity * n) + 64.0, 1.0e9);
    D.off = off;
    D.rp_off = rp_off;
    D.col_off = col_off;
    D.col_s_off = col_s_off;
    D.gram_off = gram_off;
    D.meta_off = meta_off;
    D.cell_off = cell_off;
    D.R = 0.0;
    D.ncx = D.ncx_f = 1;  // until pecc_set_radius
    D.inv_cs = 1.0;
    D.inv_f = 1.f;
    off += n;
    rp_off += 2 * (int64_t)(n + 1);
    col_off += 2 * (int64_t)D.cap;
    col_s_off += D.cap;
    gram_off += (int64_t)k * kBasis * kBasis;
    meta_off += (int64_t)k * kMetaInts;
    const int cap_c = cell_grid_cap(n);  // the cell table of the largest grid the instance can get
    cell_off += 2 * (int64_t)cap_c * cap_c + 2;
  }
  pecc_status s;
#define ALC(ptr, T, count)                                   \
  do {                                                       \
    T *tmp_ = nullptr;                                       \
    if ((s = dalloc<T>(ctx, &tmp_, (size_t)(count))) != PECC_OK) return bail(s); \
    ptr = tmp_;                                              \
  } while (0)
  ALC(ctx->desc, InstDesc, ctx->num);
  ALC(ctx->out, InstOut, ctx->num);
  ALC(ctx->order, int32_t, ctx->num);
  ALC(ctx->eorder, int32_t, ctx->num);
  ALC(ctx->queue, int32_t, 5);  // descent phases 0..3, container adjustment 4
  ALC(ctx->t0, long long, 1);
  ALC(ctx->inst_of, int32_t, total);
  ALC(ctx->x64, double2, total);
  if (!fp64) ALC(ctx->x32, float2, total);
  void *p;
  ALC(p, double2, total); ctx->xw = p;
  ALC(p, double2, total); ctx->xb = p;
  ALC(p, double2, total); ctx->xo = p;
  ALC(p, double2, total); ctx->g = p;
  ALC(p, double2, total); ctx->gt = p;
  ALC(p, double2, total); ctx->d = p;
  ALC(p, double2, total); ctx->xbuild = p;
  ALC(p, char, vec2 * (size_t)m1 * (size_t)total); ctx->S = p;
  ALC(p, char, vec2 * (size_t)m1 * (size_t)total); ctx->Y = p;
  ALC(p, char, vecs * (size_t)gram_off); ctx->gram = p;
  ALC(ctx->meta, int32_t, meta_off);
  ALC(p, double, total); ctx->ecirc = p;
  ALC(ctx->perm, int32_t, total);
  ALC(ctx->skey, uint64_t, total);
  ALC(ctx->rp, int32_t, rp_off);
  ALC(ctx->col, int32_t, col_off);
  ALC(ctx->rp_s, int32_t, total + ctx->num);
  ALC(ctx->col_s, int32_t, col_s_off);
  ALC(ctx->ckey, uint32_t, total);
  ALC(ctx->ckey_s, uint32_t, total);
  ALC(ctx->corder, int32_t, total);
  ALC(ctx->corder_s, int32_t, total);
  ALC(ctx->nnz, int64_t, ctx->num + 1);
  ALC(ctx->cells, int32_t, cell_off);
  ALC(ctx->stage, char, (size_t)ctx->num * 32);
  if (!ctx->big.empty()) {
    int occ = 0, nmax_big = 0, kmax = 1;
    const int ar = cfg->precision == PECC_FP64 ? 0 : 1;
    for (int a = ar; a <= (cfg->precision == PECC_FP32_POLISH64 ? 2 : ar); ++a) {
      int o = 0;
      if (grid_descend_occupancy(a, ctx->gblock, &o) != cudaSuccess || o < 1)
        return bail(fail(ctx, PECC_ERR_CUDA, "whole-GPU descent kernel does not fit an SM"));
      occ = occ == 0 ? o : std::min(occ, o);
    }
    ctx->ggrid = ctx->num_sms * occ;
    for (int q : ctx->big) { nmax_big = std::max(nmax_big, ctx->n[q]); kmax = std::max(kmax, ctx->k[q]); }
    ALC(ctx->gb.part, double, 2 * (size_t)ctx->ggrid * 72);  // two alternating partial buffers
    ALC(ctx->gb.res, double, 2 * 72 + 1);  // two alternating total buffers, then the time-budget flag
    ALC(ctx->gb.ipart, int32_t, ctx->ggrid);
    ALC(ctx->gb.bucket, int32_t, 2 * (size_t)(nmax_big / 4) + 4);
    ALC(ctx->gb.hash, unsigned long long, 1);
    ALC(p, char, (size_t)ctx->ggrid * kmax * kBasis * kBasis * 8); ctx->gb.gram = p;
    ctx->gb.kmax = kmax;
    ALC(ctx->gctl, GridCtl, 1);
  }
#undef ALC
  // instance of every circle, processing order (largest first)
  std::vector<int32_t> inst_of(total);
  for (int q = 0; q < ctx->num; ++q)
    std::fill(inst_of.begin() + ctx->desc_h[q].off, inst_of.begin() + ctx->desc_h[q].off + ctx->n[q], q);
  std::vector<int32_t> order(ctx->num);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctx->n[a] > ctx->n[b]; });
  if (total > 0 && cudaMemcpy(ctx->inst_of, inst_of.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice))
    return bail(fail(ctx, PECC_ERR_CUDA, "upload inst_of"));
  if (ctx->num > 0 && (cudaMemcpy(ctx->order, order.data(), sizeof(int32_t) * ctx->num, cudaMemcpyHostToDevice) ||
                       cudaMemcpy(ctx->eorder, order.data(), sizeof(int32_t) * ctx->num, cudaMemcpyHostToDevice)))
    return bail(fail(ctx, PECC_ERR_CUDA, "upload order"));
  if (ctx->num > 0 &&
      cudaMemcpy(ctx->desc, ctx->desc_h.data(), sizeof(InstDesc) * ctx->num, cudaMemcpyHostToDevice))
    return bail(fail(ctx, PECC_ERR_CUDA, "upload instance descriptors"));
  if (cudaMemset(ctx->out, 0, sizeof(InstOut) * std::max(ctx->num, 1)) ||
      cudaMemset(ctx->rp_s, 0, sizeof(int32_t) * (total + ctx->num)) ||
      cudaMemset(ctx->x64, 0, sizeof(double2) * std::max<int64_t>(total, 1)))
    return bail(fail(ctx, PECC_ERR_CUDA, "memset"));

  // launch shape
  const int arith = cfg->precision == PECC_FP64 ? 0 : 1;
  int nmax = 0;
  for (int v : ctx->n) nmax = std::max(nmax, v);
  int blk = cfg->block_threads;
  if (blk == 0) {
    int want = (nmax + 1) / 2;  // about two circles per thread
    blk = std::min(descend_max_block(arith), std::max(64, (want + 31) / 32 * 32));
    if (ctx->num > ctx->num_sms) blk = std::min(blk, 256);
  }
  ctx->block = blk;
  ctx->bps = 0;
  ctx->grid = 0;
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) return bail(fail(ctx, PECC_ERR_CUDA, "cudaEventCreate"));
  *out = ctx;
  return PECC_OK;
}

pecc_status pecc_destroy(pecc_ctx *ctx) {
  if (!ctx) return PECC_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  for (int i = 0; i < 4; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (void *p : ctx->allocs) cudaFree(p);
  delete ctx;
  return PECC_OK;
}

pecc_status pecc_selftest_grid_barrier(int64_t timeout_ns, int32_t *failed_host, int64_t *waited_ns_host) {
  if (!failed_host || !waited_ns_host || timeout_ns <= 0 || timeout_ns > 10000000000ll)
    return fail(nullptr, PECC_ERR_ARG, "pecc_selftest_grid_barrier: bad argument");
  int f = 0;
  long long w = 0;
  cudaError_t e = selftest_grid_barrier((long long)timeout_ns, &f, &w);
  if (e != cudaSuccess) return fail(nullptr, PECC_ERR_CUDA, "pecc_selftest_grid_barrier: %s", cudaGetErrorString(e));
  *failed_host = f;
  *waited_ns_host = w;
  return PECC_OK;
}

const char *pecc_last_error(pecc_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

pecc_status pecc_set_radius(pecc_ctx *ctx, const double *R_dev) {
  if (!ctx) return PECC_ERR_ARG;
  if (ctx->num == 0) return PECC_OK;
  if (!R_dev) return fail(ctx, PECC_ERR_ARG, "R_dev is NULL");
  // the radii and each instance's cell grids are written on the device, in stream order; the cell
  // tables were sized at create for the largest grid an instance can get
  CK(launch_set_radius(ctx->desc, R_dev, ctx->num, ctx->cfg.l_cut, ctx->stream));
  ctx->radius_set = true;
  ctx->radius_host_known = false;
  ctx->lists_prec = -1;
  return PECC_OK;
}

static pecc_status need_radius(pecc_ctx *ctx) {
  if (!ctx) return PECC_ERR_ARG;
  if (!ctx->radius_set && ctx->num > 0) return fail(ctx, PECC_ERR_ARG, "pecc_set_radius has not been called");
  return PECC_OK;
}

pecc_status pecc_set_positions(pecc_ctx *ctx, const double *xy_dev) {
  if (!ctx) return PECC_ERR_ARG;
  if (ctx->total > 0 && !xy_dev) return fail(ctx, PECC_ERR_ARG, "xy_dev is NULL");
  CK(launch_set_positions(sparams(ctx), xy_dev, ctx->cfg.precision == PECC_FP64 ? 0 : 1, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_init_random(pecc_ctx *ctx, uint64_t seed) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  CK(launch_init(sparams(ctx), seed, ctx->cfg.init_mode, ctx->cfg.precision == PECC_FP64 ? 0 : 1, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_get_positions(pecc_ctx *ctx, double *xy_dev) {
  if (!ctx) return PECC_ERR_ARG;
  if (ctx->total > 0 && !xy_dev) return fail(ctx, PECC_ERR_ARG, "xy_dev is NULL");
  CK(launch_get_positions(sparams(ctx), xy_dev, ctx->cfg.precision == PECC_FP32 ? 1 : 0, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_rebuild_neighbors_ex(pecc_ctx *ctx, int32_t eval, int32_t force, int32_t *rebuilt_dev) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (eval < 0 || eval > 2) return fail(ctx, PECC_ERR_ARG, "bad eval");
  int prec = eval == PECC_FP32 ? 1 : 0;
  if (prec == 1 && !ctx->x32) return fail(ctx, PECC_ERR_ARG, "FP32 lists need an FP32 context");
  if (ctx->lists_prec != prec) force = 1;
  CK(launch_build(sparams(ctx), prec, force, rebuilt_dev, nullptr, ctx->block_build, ctx->stream));
  ctx->lists_prec = prec;
  return PECC_OK;
}

pecc_status pecc_rebuild_neighbors(pecc_ctx *ctx, int32_t force, int32_t *rebuilt_dev) {
  if (!ctx) return PECC_ERR_ARG;
  return pecc_rebuild_neighbors_ex(ctx, ctx->cfg.precision == PECC_FP64 ? PECC_FP64 : PECC_FP32, force, rebuilt_dev);
}

pecc_status pecc_neighbor_count(pecc_ctx *ctx, int64_t *nnz_host) {
  if (!ctx || !nnz_host) return PECC_ERR_ARG;
  if (ctx->lists_prec < 0 && ctx->num > 0) return fail(ctx, PECC_ERR_ARG, "no neighbor lists built");
  std::vector<int64_t> v(ctx->num);
  CK(launch_nnz(sparams(ctx), ctx->nnz, ctx->stream));
  if (ctx->num) CK(cudaMemcpyAsync(v.data(), ctx->nnz, sizeof(int64_t) * ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int64_t t = 0;
  for (int q = 0; q < ctx->num; ++q) {
    if (v[q] > ctx->desc_h[q].cap) return fail(ctx, PECC_ERR_NBR_OVERFLOW, "instance %d: %lld entries over capacity %d",
                                              q, (long long)v[q], ctx->desc_h[q].cap);
    t += v[q];
  }
  *nnz_host = t;
  return PECC_OK;
}

pecc_status pecc_export_neighbors(pecc_ctx *ctx, int32_t *row_ptr_dev, int32_t *col_dev, int64_t cap) {
  int64_t nnz = 0;
  pecc_status s = pecc_neighbor_count(ctx, &nnz);
  if (s) return s;
  if (cap < nnz) return fail(ctx, PECC_ERR_ARG, "cap %lld below %lld entries", (long long)cap, (long long)nnz);
  if (!row_ptr_dev || (nnz > 0 && !col_dev)) return fail(ctx, PECC_ERR_ARG, "NULL output");
  std::vector<int64_t> v(ctx->num), base(ctx->num + 1, 0);
  if (ctx->num) CK(cudaMemcpyAsync(v.data(), ctx->nnz, sizeof(int64_t) * ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < ctx->num; ++q) base[q + 1] = base[q] + v[q];
  int64_t *dbase = nullptr;
  CK(cudaMalloc(&dbase, sizeof(int64_t) * (ctx->num + 1)));
  cudaError_t e = cudaMemcpyAsync(dbase, base.data(), sizeof(int64_t) * (ctx->num + 1), cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess) e = launch_export_csr(sparams(ctx), dbase, row_ptr_dev, col_dev, ctx->stream);
  const cudaError_t es = cudaStreamSynchronize(ctx->stream);  // base[] and dbase live until here
  cudaFree(dbase);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return fail(ctx, PECC_ERR_CUDA, "export: %s", cudaGetErrorString(e));
  return PECC_OK;
}

pecc_status pecc_export_cells(pecc_ctx *ctx, uint32_t *key_dev, int32_t *order_dev) {
  if (!ctx) return PECC_ERR_ARG;
  if (ctx->lists_prec < 0 && ctx->num > 0) return fail(ctx, PECC_ERR_ARG, "no neighbor lists built");
  if (ctx->total > 0 && (!key_dev || !order_dev)) return fail(ctx, PECC_ERR_ARG, "NULL output");
  CK(launch_export_cells(sparams(ctx), key_dev, order_dev, ctx->stream));
  return PECC_OK;
}

// Which energy + gradient kernels a call needs: the largest instance the block kernel stages, and
// whether any instance is too large for it.
static void energy_grad_split(const pecc_ctx *ctx, int eval, int *max_small_n, bool *any_large) {
  const int lim = energy_stage_n(eval);
  *max_small_n = -1;  // no instance for the block kernel
  *any_large = false;
  for (int q = 0; q < ctx->num; ++q) {
    if (ctx->n[q] <= lim) *max_small_n = std::max(*max_small_n, ctx->n[q]);
    else *any_large = true;
  }
}

static cudaError_t energy_grad_launch(pecc_ctx *ctx, const StandaloneParams &sp, int eval, double *E, void *grad) {
  int ms = 0;
  bool big = false;
  energy_grad_split(ctx, eval, &ms, &big);
  return launch_energy_grad(sp, eval, E, grad, ctx->ecirc, ms, big, ctx->stream);
}

pecc_status pecc_energy_grad_ex(pecc_ctx *ctx, int32_t eval, double *E_dev, void *grad_dev) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (eval < 0 || eval > 2) return fail(ctx, PECC_ERR_ARG, "bad eval");
  int prec = eval == PECC_FP32 ? 1 : 0;
  if (ctx->lists_prec != prec) return fail(ctx, PECC_ERR_ARG, "neighbor lists were not built for this arithmetic");
  if (ctx->total > 0 && (!E_dev || !grad_dev)) return fail(ctx, PECC_ERR_ARG, "NULL output");
  if (eval == PECC_FP32_POLISH64 && ctx->cfg.precision == PECC_FP64)
    return fail(ctx, PECC_ERR_ARG, "the mixed arithmetic needs an FP32 context");
  CK(energy_grad_launch(ctx, sparams(ctx), eval, E_dev, grad_dev));
  return PECC_OK;
}

pecc_status pecc_energy_grad(pecc_ctx *ctx, double *E_dev, void *grad_dev) {
  if (!ctx) return PECC_ERR_ARG;
  return pecc_energy_grad_ex(ctx, ctx->cfg.precision == PECC_FP64 ? PECC_FP64 : PECC_FP32, E_dev, grad_dev);
}

// Launch shape of one descent arithmetic.  block / bps_target 0 = the config's, else the default:
// about two circles per thread (at most 256 threads when instances outnumber SMs) and as many
// blocks per SM as fit.
// Dynamic shared memory: the largest working set, capped so that bps_target blocks share an SM
// (the working set spills to global memory past the cap); blocks per SM from the occupancy
// calculator.
static pecc_status plan_launch(pecc_ctx *ctx, int arith, int block = 0, int bps_target = 0) {
  pecc_ctx::Launch &L = ctx->lc[arith];
  int dev = ctx->device, optin = 0, per_sm = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const bool many = ctx->num > ctx->num_sms;
  int blk = block > 0 ? block : ctx->cfg.block_threads;
  if (blk == 0) {
    int nmax = 0;
    for (int q = 0; q < ctx->num; ++q)
      if (!ctx->desc_h[q].big) nmax = std::max(nmax, ctx->n[q]);
    int want = (nmax + 1) / 2;
    blk = std::min(descend_max_block(arith), std::max(64, (want + 31) / 32 * 32));
    if (many) blk = std::min(blk, 256);
  }
  blk = std::min(blk, descend_max_block(arith));
  L.block = blk;
  size_t need = 0, mand = 0;
  for (int q = 0; q < ctx->num; ++q) {
    const InstDesc &D = ctx->desc_h[q];
    if (D.big) continue;
    for (int a = (arith == 3 ? 1 : arith); a <= (arith == 3 ? 2 : arith); ++a) {  // fused: both phases
      int k = D.k;
      if (a == 2 && ctx->cfg.polish_k > 0) k = std::min(ctx->cfg.polish_k, D.k);
      // the grid's size is known on the device only: plan for the largest it can be
      need = std::max(need, descend_smem_need(a, D.n, k, cell_grid_cap(D.n), blk, ctx->cfg.lbfgs_m,
                                                   ctx->cfg.list_outer > 0.0));
      mand = std::max(mand, descend_smem_mandatory(a, k, blk));
    }
  }
  if (bps_target <= 0) bps_target = ctx->cfg.blocks_per_sm;
  const bool fixed = bps_target > 0;  // else as many blocks per SM as fit
  if (!fixed) bps_target = many ? 2 : 1;
  // the compiled instance: the largest register budget that reaches the target blocks per SM (the
  // most resident blocks when none does); without a target, the largest budget
  const DescendVariant *vs = nullptr;
  const int nv = descend_variants(arith, &vs);
  int best = -1, best_occ = 0;
  size_t best_smem = 0;
  for (int v = 0; v < nv; ++v) {
    if (blk > vs[v].max_threads) continue;
    // per-block share: the SM's shared memory over the target, in whole KB (allocation
    // granularity), less the static block state and the 1 KB the system reserves per block
    const size_t stat = (vs[v].static_smem + 1024 + 255) & ~size_t(255);
    size_t cap = ((size_t)per_sm / bps_target) & ~size_t(1023);
    cap = (cap > stat ? cap - stat : 0);
    cap = std::min(cap, (size_t)optin - stat);
    if (ctx->cfg.smem_per_block > 0) cap = std::min(cap, (size_t)ctx->cfg.smem_per_block);
    const size_t smem = std::max(mand, std::min(need, cap) & ~size_t(255));
    if (smem + stat > (size_t)optin) continue;
    CK(cudaFuncSetAttribute(vs[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vs[v].fn, blk, smem));
    if (occ < 1) continue;
    if (best < 0 || occ > best_occ) { best = v; best_occ = occ; best_smem = smem; }
    if (!fixed || occ >= bps_target) break;
  }
  if (best < 0)
    return fail(ctx, PECC_ERR_ARG, "descent kernel does not fit an SM (block %d, %zu bytes of shared memory needed)", blk, mand);
  CK(cudaFuncSetAttribute(vs[best].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_smem));
  L.var = best;
  L.smem = best_smem;
  L.bps = fixed ? std::min(bps_target, best_occ) : best_occ;
  L.grid = (int)std::min<int64_t>(ctx->num, (int64_t)ctx->num_sms * L.bps);
  return PECC_OK;
}

static const DescendVariant &variant_of(pecc_ctx *c, int arith) {
  const DescendVariant *vs = nullptr;
  descend_variants(arith, &vs);
  return vs[c->lc[arith].var];
}

static DescendParams dparams(pecc_ctx *c, int phase) {
  DescendParams p{};
  p.desc = c->desc;
  p.out = c->out;
  p.num = c->num;
  p.num_dev = c->num_dev;
  p.order = c->order;
  p.queue = c->queue + phase;
  p.x32 = c->x32;
  p.x64 = c->x64;
  p.xw = c->xw; p.xb = c->xb; p.xo = c->xo;
  p.g = c->g; p.gt = c->gt; p.d = c->d;
  p.S = c->S; p.Y = c->Y;
  p.perm = c->perm;
  p.skey = c->skey;
  p.rp = c->rp; p.col = c->col;
  p.ckey = c->ckey; p.corder = c->corder; p.cells = c->cells;
  p.gram = c->gram; p.meta = c->meta;
  const pecc_config &f = c->cfg;
  p.l_cut = f.l_cut; p.rebuild_disp = f.rebuild_disp; p.step_max = f.step_max;
  p.e_tol = f.e_tol; p.gsum_tol = f.gsum_tol; p.c1 = f.c1; p.curv_eps = f.curv_eps; p.polish_gate = f.polish_gate;
  p.m = f.lbfgs_m; p.max_iter = f.max_iter; p.max_trials = f.max_trials; p.anm = f.anm; p.partition = f.partition;
  p.part_seed = f.partition_seed;
  p.list_outer = f.list_outer;
  p.stall_rel = (phase == 2) ? f.polish_stall_rel : f.stall_rel;
  p.stall_window = (phase == 2) ? f.polish_stall_window : f.stall_window;
  p.t0 = c->t0;
  p.budget_ns = f.time_budget_ns;
  p.k_override = (phase == 2) ? f.polish_k : 0;
  p.smem_bytes = c->lc[phase].smem;
  if (phase <= 1 && c->dump_cnt) {  // the first phase only: FP64, or the FP32 descent
    p.dump_cnt = c->dump_cnt;
    p.dump_col = c->dump_col;
    p.dump_xb = (double2 *)c->dump_xb;
    p.dump_stride = c->dump_stride;
  }
  return p;
}

// The whole descent as one stream-ordered sequence (captured into a CUDA graph once).
static cudaError_t enqueue_descend(pecc_ctx *c) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->queue, 0, 4 * sizeof(int32_t), c->stream))) return e;
  if ((e = launch_stamp(c->t0, c->stream))) return e;
  if ((e = cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal))) return e;
  if (c->cfg.precision == PECC_FP64) {
    if ((e = launch_descend(variant_of(c, 0), dparams(c, 0), c->lc[0].grid, c->lc[0].block, c->stream))) return e;
    if ((e = cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal))) return e;
    return cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal);
  }
  if (c->cfg.precision == PECC_FP32_POLISH64 && c->cfg.fuse_phases) {
    DescendParams p32 = dparams(c, 1), p64 = dparams(c, 2);
    p64.max_iter = c->cfg.polish_max_iter;
    p32.smem_bytes = p64.smem_bytes = c->lc[3].smem;
    if ((e = launch_descend_fused(variant_of(c, 3), p32, p64, c->lc[3].grid, c->lc[3].block, c->stream))) return e;
    if ((e = cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal))) return e;
    return cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal);
  }
  if ((e = launch_descend(variant_of(c, 1), dparams(c, 1), c->lc[1].grid, c->lc[1].block, c->stream))) return e;
  if ((e = cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal))) return e;
  if (c->cfg.precision == PECC_FP32_POLISH64) {
    DescendParams p = dparams(c, 2);
    p.max_iter = c->cfg.polish_max_iter;
    if ((e = launch_descend(variant_of(c, 2), p, c->lc[2].grid, c->lc[2].block, c->stream))) return e;
  }
  return cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal);
}

static pecc_status descend_dense(pecc_ctx *ctx, int32_t *iters_dev, int32_t *status_dev) {
  for (int q = 0; q < ctx->num; ++q)
    if (ctx->desc_h[q].big) return fail(ctx, PECC_ERR_ARG, "qn_dense: instance %d has 16384 circles or more", q);
  if (!ctx->denseH) {
    std::vector<int64_t> off(ctx->num);
    int64_t words = 0;
    for (int q = 0; q < ctx->num; ++q) {
      off[q] = words;
      words += dense_h_words(ctx->n[q], ctx->k[q]);
    }
    pecc_status s;
    if ((s = dalloc<double>(ctx, &ctx->denseH, (size_t)std::max<int64_t>(words, 1)))) return s;
    if ((s = dalloc<int64_t>(ctx, &ctx->dense_hoff, ctx->num))) return s;
    CK(cudaMemcpyAsync(ctx->dense_hoff, off.data(), sizeof(int64_t) * ctx->num, cudaMemcpyHostToDevice, ctx->stream));
  }
  DenseParams p{};
  p.desc = ctx->desc; p.out = ctx->out; p.num = ctx->num; p.order = ctx->order; p.queue = ctx->queue;
  p.x = ctx->x64;
  p.g = (double2 *)ctx->g; p.gn = (double2 *)ctx->gt; p.d = (double2 *)ctx->d; p.xo = (double2 *)ctx->xo;
  p.xb = (double2 *)ctx->xb; p.xs = (double2 *)ctx->xbuild; p.hy = (double2 *)ctx->xw;
  p.skey = ctx->skey; p.perm = ctx->perm; p.batch_of = (int32_t *)ctx->ckey_s;
  p.rp = ctx->rp; p.col = ctx->col; p.ckey = ctx->ckey; p.corder = ctx->corder; p.cells = ctx->cells;
  p.H = ctx->denseH; p.h_off = ctx->dense_hoff;
  const pecc_config &f = ctx->cfg;
  p.l_cut = f.l_cut; p.rebuild_disp = f.rebuild_disp; p.step_max = f.step_max; p.e_tol = f.e_tol;
  p.gsum_tol = f.gsum_tol; p.c1 = f.c1; p.curv_eps = f.curv_eps;
  p.max_iter = f.max_iter; p.max_trials = f.max_trials; p.anm = f.anm; p.partition = f.partition;
  p.part_seed = f.partition_seed;
  if (!ctx->ev[0])
    for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&ctx->ev[i]));
  CK(cudaMemsetAsync(ctx->queue, 0, sizeof(int32_t), ctx->stream));
  CK(cudaEventRecord(ctx->ev[0], ctx->stream));
  CK(launch_dense(p, (int)std::min<int64_t>(ctx->num, (int64_t)ctx->num_sms * 2), ctx->stream));
  CK(cudaEventRecord(ctx->ev[1], ctx->stream));
  CK(cudaEventRecord(ctx->ev[2], ctx->stream));
  ctx->dense_ran = true;
  ctx->lists_prec = -1;
  if (iters_dev || status_dev)
    CK(launch_outputs(ctx->out, ctx->num, iters_dev, status_dev, nullptr, nullptr, nullptr, nullptr, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_descend(pecc_ctx *ctx, int32_t *iters_dev, int32_t *status_dev) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (ctx->num == 0) return PECC_OK;
  if (ctx->cfg.qn_dense) return descend_dense(ctx, iters_dev, status_dev);
  for (int q = 0; q < ctx->num; ++q)
    if (ctx->n[q] > 65535 && !ctx->desc_h[q].big)
      return fail(ctx, PECC_ERR_ARG, "pecc_descend: instance %d has more than 65535 circles", q);
  if (!ctx->lc_ready) {
    const int pr = ctx->cfg.precision;
    const int tb = ctx->tuned ? ctx->tuned_block : 0, tt = ctx->tuned ? ctx->tuned_bps : 0;
    if (pr == PECC_FP64) {
      if ((s = plan_launch(ctx, 0, tb, tt))) return s;
    } else if (pr == PECC_FP32_POLISH64 && ctx->cfg.fuse_phases) {
      if ((s = plan_launch(ctx, 3, tb > 0 ? std::min(tb, 256) : 0, tt))) return s;
    } else {
      if ((s = plan_launch(ctx, 1, tb, tt))) return s;
      if (pr == PECC_FP32_POLISH64 && (s = plan_launch(ctx, 2, tb > 0 ? std::min(tb, 256) : 0, tt))) return s;
    }
    ctx->lc_ready = true;
  }
  if (!ctx->graph) {
    cudaStream_t cs = ctx->stream;
    bool own = false;
    if (!cs) {  // capture needs a non-legacy stream
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    cudaGraph_t graph = nullptr;
    cudaStream_t saved = ctx->stream;
    ctx->stream = cs;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_descend(ctx);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    ctx->stream = saved;
    if (own) cudaStreamDestroy(cs);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(ctx, PECC_ERR_CUDA, "capture: %s", cudaGetErrorString(e ? e : e2));
    }
    e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, PECC_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
  }
  CK(cudaGraphLaunch(ctx->graph, ctx->stream));
  // large instances: one cooperative whole-GPU launch per instance and phase
  for (int q : ctx->big) {
    if (ctx->cfg.precision == PECC_FP64) {
      CK(launch_grid_descend(0, dparams(ctx, 0), q, ctx->gb, ctx->gctl, ctx->ggrid, ctx->gblock, ctx->stream));
    } else {
      CK(launch_grid_descend(1, dparams(ctx, 1), q, ctx->gb, ctx->gctl, ctx->ggrid, ctx->gblock, ctx->stream));
      if (ctx->cfg.precision == PECC_FP32_POLISH64) {
        DescendParams p2 = dparams(ctx, 2);
        p2.max_iter = ctx->cfg.polish_max_iter;
        CK(launch_grid_descend(2, p2, q, ctx->gb, ctx->gctl, ctx->ggrid, ctx->gblock, ctx->stream));
      }
    }
  }
  ctx->lists_prec = -1;  // the descent reuses the scratch the standalone lists rely on
  if (iters_dev || status_dev)
    CK(launch_outputs(ctx->out, ctx->num, iters_dev, status_dev, nullptr, nullptr, nullptr, nullptr, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_set_list_dump(pecc_ctx *ctx, int32_t stride, int32_t *cnt_dev, int32_t *col_dev, double *xb_dev) {
  if (!ctx) return PECC_ERR_ARG;
  if (cnt_dev && (stride < 1 || !col_dev || !xb_dev))
    return fail(ctx, PECC_ERR_ARG, "pecc_set_list_dump: stride must be >= 1 with col_dev and xb_dev set");
  ctx->dump_cnt = cnt_dev;
  ctx->dump_col = cnt_dev ? col_dev : nullptr;
  ctx->dump_xb = cnt_dev ? xb_dev : nullptr;
  ctx->dump_stride = cnt_dev ? stride : 0;
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }  // captured again
  return PECC_OK;
}

pecc_status pecc_get_energy(pecc_ctx *ctx, double *E_dev) {
  if (!ctx || (ctx->num > 0 && !E_dev)) return PECC_ERR_ARG;
  CK(launch_outputs(ctx->out, ctx->num, nullptr, nullptr, E_dev, nullptr, nullptr, nullptr, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_get_counters(pecc_ctx *ctx, int32_t *builds_dev, int32_t *changes_dev, int32_t *trials_dev) {
  if (!ctx) return PECC_ERR_ARG;
  CK(launch_outputs(ctx->out, ctx->num, nullptr, nullptr, nullptr, builds_dev, changes_dev, trials_dev, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_autotune(pecc_ctx *ctx, int32_t sweeps, uint64_t seed, int32_t *block_out, int32_t *bps_out) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (sweeps < 1) return fail(ctx, PECC_ERR_ARG, "sweeps must be >= 1");
  if (ctx->num == 0) return PECC_OK;
  const int arith = ctx->cfg.precision == PECC_FP64 ? 0 : 1;
  const int plan_arith = (ctx->cfg.precision == PECC_FP32_POLISH64 && ctx->cfg.fuse_phases) ? 3 : arith;
  // keep the caller's coordinates (both copies, bit for bit) and restore them afterwards
  const size_t b64 = sizeof(double2) * (size_t)ctx->total, b32 = ctx->x32 ? sizeof(float2) * (size_t)ctx->total : 0;
  char *saved = nullptr;
  CK(cudaMalloc(&saved, std::max<size_t>(b64 + b32, 16)));
  CK(cudaMemcpyAsync(saved, ctx->x64, b64, cudaMemcpyDeviceToDevice, ctx->stream));
  if (b32) CK(cudaMemcpyAsync(saved + b64, ctx->x32, b32, cudaMemcpyDeviceToDevice, ctx->stream));
  const pecc_config keep = ctx->cfg;
  ctx->cfg.max_iter = sweeps;
  ctx->cfg.stall_window = 0;
  ctx->cfg.precision = arith == 1 ? PECC_FP32 : PECC_FP64;
  const int blocks[3] = {128, 256, 512};
  const int targets[5] = {1, 2, 4, 5, 6};
  double best = -1.0;
  int best_b = 0, best_t = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<int32_t> st((size_t)ctx->num * 10);
  pecc_status err = PECC_OK;
  for (int bi = 0; bi < 3 && !err; ++bi) {
    for (int ti = 0; ti < 5 && !err; ++ti) {
      // shapes the planned kernel can run; the fused kernel's 512-thread instance serves launches of
      // a few instances (its default plan), not the many-instance shapes searched here
      if (blocks[bi] > (plan_arith == 3 ? 256 : descend_max_block(plan_arith))) continue;
      if ((err = plan_launch(ctx, arith, blocks[bi], targets[ti]))) break;
      if (ctx->lc[arith].bps < targets[ti]) continue;  // that many blocks do not fit an SM
      ctx->lc_ready = true;
      if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
      if ((err = pecc_init_random(ctx, seed))) break;
      cudaEventRecord(e0, ctx->stream);
      if ((err = pecc_descend(ctx, nullptr, nullptr))) break;
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { err = fail(ctx, PECC_ERR_CUDA, "autotune sync"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      // circle-sweeps per second: sum over instances of n x sweeps done
      int32_t *dstats = nullptr;
      if (cudaMalloc(&dstats, sizeof(int32_t) * 10 * ctx->num) != cudaSuccess) { err = fail(ctx, PECC_ERR_OOM, "autotune"); break; }
      cudaError_t ce = launch_stats(ctx->out, ctx->num, dstats, ctx->stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(st.data(), dstats, sizeof(int32_t) * 10 * ctx->num, cudaMemcpyDeviceToHost, ctx->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
      cudaFree(dstats);
      if (ce != cudaSuccess) { err = fail(ctx, PECC_ERR_CUDA, "autotune stats: %s", cudaGetErrorString(ce)); break; }
      double work = 0.0;
      for (int q = 0; q < ctx->num; ++q) work += (double)ctx->n[q] * st[(size_t)q * 10 + 0];
      const double rate = work / std::max(1e-3, (double)ms);
      if (rate > best) { best = rate; best_b = blocks[bi]; best_t = targets[ti]; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->cfg = keep;
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
  ctx->lc_ready = false;  // a failed or empty search leaves the default shapes to the next descent
  if (!err && best_b > 0) {
    ctx->tuned = true;
    ctx->tuned_block = best_b;
    ctx->tuned_bps = best_t;
  }
  cudaError_t ce = cudaMemcpyAsync(ctx->x64, saved, b64, cudaMemcpyDeviceToDevice, ctx->stream);
  if (ce == cudaSuccess && b32) ce = cudaMemcpyAsync(ctx->x32, saved + b64, b32, cudaMemcpyDeviceToDevice, ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  cudaFree(saved);
  if (err) return err;
  if (ce != cudaSuccess) return fail(ctx, PECC_ERR_CUDA, "autotune restore: %s", cudaGetErrorString(ce));
  if (block_out) *block_out = best_b;
  if (bps_out) *bps_out = best_t;
  return PECC_OK;
}

pecc_status pecc_adjust_container(pecc_ctx *ctx, double *R_dev, double lambda0, int32_t rounds, int32_t *iters_dev,
                                  int32_t *status_dev, int32_t *stats_dev) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (ctx->num == 0) return PECC_OK;
  if (!R_dev || !iters_dev || !status_dev) return fail(ctx, PECC_ERR_ARG, "pecc_adjust_container: NULL pointer");
  if (rounds < 0 || !(lambda0 >= 0.0) || !std::isfinite(lambda0))
    return fail(ctx, PECC_ERR_ARG, "pecc_adjust_container: rounds must be >= 0 and lambda0 finite and >= 0");
  if (ctx->cfg.lbfgs_m > adjust_max_m()) return fail(ctx, PECC_ERR_ARG, "pecc_adjust_container: lbfgs_m too large");
  const size_t slots = (size_t)adjust_max_m() * (size_t)std::max<int64_t>(ctx->total, 1);
  if (!ctx->adjS) {
    if ((s = dalloc<double2>(ctx, &ctx->adjS, slots))) return s;
    if ((s = dalloc<double2>(ctx, &ctx->adjY, slots))) return s;
  }
  AdjustParams p{};
  p.desc = ctx->desc;
  p.num = ctx->num;
  p.from32 = ctx->cfg.precision == PECC_FP32 ? 1 : 0;
  p.x32 = ctx->x32;
  p.x64 = ctx->x64;
  p.R = R_dev;
  p.g = (double2 *)ctx->g; p.gn = (double2 *)ctx->gt; p.d = (double2 *)ctx->d; p.zo = (double2 *)ctx->xo;
  p.xb = (double2 *)ctx->xw; p.xs = (double2 *)ctx->xbuild; p.sv = (double2 *)ctx->xb;
  p.S = ctx->adjS; p.Y = ctx->adjY;
  p.rp = ctx->rp; p.col = ctx->col; p.ckey = ctx->ckey; p.corder = ctx->corder; p.cells = ctx->cells;
  p.iters = iters_dev; p.status = status_dev; p.queue = ctx->queue + 4; p.stats = stats_dev;
  const pecc_config &f = ctx->cfg;
  p.l_cut = f.l_cut; p.rebuild_disp = f.rebuild_disp; p.step_max = f.step_max; p.gsum_tol = f.gsum_tol;
  p.c1 = f.c1; p.curv_eps = f.curv_eps; p.lambda0 = lambda0;
  p.m = f.lbfgs_m; p.max_iter = f.max_iter; p.max_trials = f.max_trials; p.anm = f.anm; p.rounds = rounds;
  CK(cudaMemsetAsync(ctx->queue + 4, 0, sizeof(int32_t), ctx->stream));
  const int mixed = ctx->cfg.precision == PECC_FP64 ? 0 : 1;
  CK(launch_adjust(p, mixed, (int)std::min<int64_t>(ctx->num, (int64_t)ctx->num_sms * 4), ctx->stream));
  ctx->lists_prec = -1;  // the standalone lists' reference coordinates served as scratch
  return PECC_OK;
}

pecc_status pecc_get_stats(pecc_ctx *ctx, int32_t *stats_dev) {
  if (!ctx || (ctx->num > 0 && !stats_dev)) return PECC_ERR_ARG;
  CK(launch_stats(ctx->out, ctx->num, stats_dev, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_phase_times(pecc_ctx *ctx, float *ms_host) {
  if (!ctx || !ms_host) return PECC_ERR_ARG;
  if (!ctx->graph && !ctx->dense_ran) return fail(ctx, PECC_ERR_ARG, "pecc_descend has not run");
  CK(cudaEventSynchronize(ctx->ev[2]));
  float a = 0.f, b = 0.f, c = 0.f;
  CK(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
  CK(cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]));
  CK(cudaEventElapsedTime(&c, ctx->ev[0], ctx->ev[2]));
  ms_host[0] = a;
  ms_host[1] = b;
  ms_host[2] = c;
  return PECC_OK;
}

pecc_status pecc_get_launch(pecc_ctx *ctx, int32_t *block_threads, int32_t *blocks_per_sm, int32_t *grid) {
  if (!ctx) return PECC_ERR_ARG;
  const int a = ctx->cfg.precision == PECC_FP64 ? 0
                : (ctx->cfg.precision == PECC_FP32_POLISH64 && ctx->cfg.fuse_phases ? 3 : 1);
  if (block_threads) *block_threads = ctx->lc[a].block;
  if (blocks_per_sm) *blocks_per_sm = ctx->lc[a].bps;
  if (grid) *grid = ctx->lc[a].grid;
  return PECC_OK;
}

// ------------------------------------------------------------------------------ learned part ----
struct pecc_mlp {
  float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *part = nullptr, *lpart = nullptr;
  __nv_bfloat16 *wb = nullptr;
  int step = 0, sms = 1;
  cudaStream_t stream = nullptr;
  std::string err;
};

static pecc_status mfail(pecc_mlp *m, pecc_status s, const char *msg) {
  if (m) m->err = msg;
  set_global_error(msg);
  return s;
}
#define MCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return mfail(mlp, PECC_ERR_CUDA, cudaGetErrorString(e_));           \
  } while (0)

int32_t pecc_mlp_num_params(void) { return mlp_num_params(); }

pecc_status pecc_mlp_destroy(pecc_mlp *mlp) {
  if (!mlp) return PECC_OK;
  cudaStreamSynchronize(mlp->stream);
  for (void *p : {(void *)mlp->params, (void *)mlp->m, (void *)mlp->v, (void *)mlp->grad, (void *)mlp->part,
                  (void *)mlp->lpart, (void *)mlp->wb})
    if (p) cudaFree(p);
  delete mlp;
  return PECC_OK;
}

pecc_status pecc_mlp_create(uint64_t seed, void *stream, pecc_mlp **out) {
  if (!out) return mfail(nullptr, PECC_ERR_ARG, "out is NULL");
  *out = nullptr;
  pecc_mlp *mlp = new pecc_mlp();
  mlp->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mlp->sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t np = (size_t)mlp_num_params();
  const int nb = mlp_train_blocks(mlp->sms);
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&mlp->params, np * 4);
  e = e ? e : cudaMalloc(&mlp->m, np * 4);
  e = e ? e : cudaMalloc(&mlp->v, np * 4);
  e = e ? e : cudaMalloc(&mlp->grad, np * 4);
  e = e ? e : cudaMalloc(&mlp->part, np * 4 * (size_t)nb);
  e = e ? e : cudaMalloc(&mlp->lpart, 4 * (size_t)nb);
  e = e ? e : cudaMalloc(&mlp->wb, 2 * (size_t)mlp_num_bf16());
  e = e ? e : cudaMemsetAsync(mlp->m, 0, np * 4, mlp->stream);
  e = e ? e : cudaMemsetAsync(mlp->v, 0, np * 4, mlp->stream);
  e = e ? e : mlp_init(mlp->params, mlp->wb, seed, mlp->stream);
  if (e != cudaSuccess) {
    pecc_status st = mfail(mlp, e == cudaErrorMemoryAllocation ? PECC_ERR_OOM : PECC_ERR_CUDA, cudaGetErrorString(e));
    pecc_mlp_destroy(mlp);
    return st;
  }
  *out = mlp;
  return PECC_OK;
}

pecc_status pecc_mlp_get_params(pecc_mlp *mlp, float *params_dev) {
  if (!mlp || !params_dev) return PECC_ERR_ARG;
  MCK(cudaMemcpyAsync(params_dev, mlp->params, 4 * (size_t)mlp_num_params(), cudaMemcpyDeviceToDevice, mlp->stream));
  return PECC_OK;
}

pecc_status pecc_mlp_set_params(pecc_mlp *mlp, const float *params_dev) {
  if (!mlp || !params_dev) return PECC_ERR_ARG;
  MCK(cudaMemcpyAsync(mlp->params, params_dev, 4 * (size_t)mlp_num_params(), cudaMemcpyDeviceToDevice, mlp->stream));
  MCK(mlp_sync_bf16(mlp->params, mlp->wb, mlp->stream));
  return PECC_OK;
}

pecc_status pecc_mlp_forward(pecc_mlp *mlp, const float *feat_dev, int64_t rows, float *out_dev) {
  if (!mlp || rows < 0 || (rows > 0 && (!feat_dev || !out_dev))) return mfail(mlp, PECC_ERR_ARG, "bad arguments");
  MCK(mlp_forward(mlp->wb, mlp->params, feat_dev, rows, out_dev, mlp->sms, mlp->stream));
  return PECC_OK;
}

pecc_status pecc_mlp_grad(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                          float *grad_dev, float *loss_dev) {
  if (!mlp || rows <= 0 || !feat_dev || !target_dev || !grad_dev) return mfail(mlp, PECC_ERR_ARG, "bad arguments");
  MCK(mlp_grad(mlp->wb, mlp->params, feat_dev, target_dev, rows, mlp->part, mlp->lpart, grad_dev, loss_dev,
               mlp->sms, mlp->stream));
  return PECC_OK;
}

pecc_status pecc_mlp_forward_trace(pecc_mlp *mlp, const float *feat_dev, int64_t rows, float *out_dev,
                                   float *trace_dev) {
  if (!mlp || rows < 0 || (rows > 0 && (!feat_dev || !out_dev || !trace_dev)))
    return mfail(mlp, PECC_ERR_ARG, "bad arguments");
  MCK(mlp_forward(mlp->wb, mlp->params, feat_dev, rows, out_dev, mlp->sms, mlp->stream, trace_dev));
  return PECC_OK;
}

pecc_status pecc_mlp_grad_trace(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                                float *grad_dev, float *loss_dev, float *fwd_trace_dev, float *bwd_trace_dev) {
  if (!mlp || rows <= 0 || !feat_dev || !target_dev || !grad_dev || !fwd_trace_dev || !bwd_trace_dev)
    return mfail(mlp, PECC_ERR_ARG, "bad arguments");
  MCK(mlp_grad(mlp->wb, mlp->params, feat_dev, target_dev, rows, mlp->part, mlp->lpart, grad_dev, loss_dev,
               mlp->sms, mlp->stream, fwd_trace_dev, bwd_trace_dev));
  return PECC_OK;
}

pecc_status pecc_mlp_train_step(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                                float lr, float *loss_dev) {
  if (!mlp || rows <= 0 || !feat_dev || !target_dev || !(lr > 0.f)) return mfail(mlp, PECC_ERR_ARG, "bad arguments");
  MCK(mlp_grad(mlp->wb, mlp->params, feat_dev, target_dev, rows, mlp->part, mlp->lpart, mlp->grad, loss_dev,
               mlp->sms, mlp->stream));
  ++mlp->step;
  MCK(mlp_adam(mlp->params, mlp->m, mlp->v, mlp->grad, mlp->wb, lr, mlp->step, mlp->stream));
  return PECC_OK;
}

static pecc_status need_fp32(pecc_ctx *ctx) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  if (!ctx->x32) return fail(ctx, PECC_ERR_ARG, "the learned warm start needs an FP32 context");
  return PECC_OK;
}

static pecc_status mlp_scratch(pecc_ctx *ctx) {
  if (ctx->feat) return PECC_OK;
  const size_t N = (size_t)std::max<int64_t>(ctx->total, 1), I = (size_t)std::max(ctx->num, 1);
  float *f = nullptr, *d = nullptr;
  float2 *b = nullptr;
  double *eb = nullptr, *ea = nullptr;
  if (cudaMalloc(&f, N * 25 * 4) || cudaMalloc(&d, N * 2 * 4) || cudaMalloc(&b, N * sizeof(float2)) ||
      cudaMalloc(&eb, I * 8) || cudaMalloc(&ea, I * 8))
    return fail(ctx, PECC_ERR_OOM, "warm-start scratch");
  for (void *p : {(void *)f, (void *)d, (void *)b, (void *)eb, (void *)ea}) ctx->allocs.push_back(p);
  ctx->feat = f; ctx->dout = d; ctx->backup = b; ctx->Eb = eb; ctx->Ea = ea;
  return PECC_OK;
}

pecc_status pecc_features(pecc_ctx *ctx, const float *unused, float *feat_dev) {
  (void)unused;
  pecc_status s = need_fp32(ctx);
  if (s) return s;
  if (ctx->total > 0 && !feat_dev) return fail(ctx, PECC_ERR_ARG, "feat_dev is NULL");
  CK(mlp_features(sparams(ctx), feat_dev, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_targets(pecc_ctx *ctx, const double *xbefore_dev, float *target_dev) {
  pecc_status s = need_fp32(ctx);
  if (s) return s;
  if (ctx->total > 0 && (!xbefore_dev || !target_dev)) return fail(ctx, PECC_ERR_ARG, "NULL pointer");
  CK(mlp_targets(sparams(ctx), xbefore_dev, target_dev, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_warm_start(pecc_ctx *ctx, pecc_mlp *mlp, int32_t rounds, int32_t *accepted_dev) {
  return pecc_warm_start_ex(ctx, mlp, rounds, 0.25, accepted_dev);
}

pecc_status pecc_warm_start_ex(pecc_ctx *ctx, pecc_mlp *mlp, int32_t rounds, double max_move, int32_t *accepted_dev) {
  pecc_status s = need_fp32(ctx);
  if (s) return s;
  if (!mlp || rounds < 0 || !(max_move > 0.0) || !(max_move <= 1e6))
    return fail(ctx, PECC_ERR_ARG, "bad arguments");
  if ((s = mlp_scratch(ctx))) return s;
  StandaloneParams sp = sparams(ctx);
  for (int r = 0; r < rounds; ++r) {
    CK(launch_build(sp, 1, 1, nullptr, nullptr, ctx->block_build, ctx->stream));
    CK(energy_grad_launch(ctx, sp, 1, ctx->Eb, ctx->g));
    CK(mlp_features(sp, ctx->feat, ctx->stream));
    CK(mlp_forward(mlp->wb, mlp->params, ctx->feat, ctx->total, ctx->dout, mlp->sms, ctx->stream));
    CK(mlp_apply(sp, ctx->dout, ctx->backup, (float)max_move, ctx->stream));
    CK(launch_build(sp, 1, 1, nullptr, nullptr, ctx->block_build, ctx->stream));
    CK(energy_grad_launch(ctx, sp, 1, ctx->Ea, ctx->g));
    CK(mlp_revert(sp, ctx->backup, ctx->Eb, ctx->Ea, accepted_dev, ctx->stream));
  }
  ctx->lists_prec = -1;
  return PECC_OK;
}

pecc_status pecc_check_feasible(pecc_ctx *ctx, double tol, uint8_t *feasible_dev, double *max_overlap_dev) {
  pecc_status s = need_radius(ctx);
  if (s) return s;
  CK(launch_feasible(sparams(ctx), ctx->cfg.precision == PECC_FP32 ? 1 : 0, tol, feasible_dev, max_overlap_dev,
                     ctx->block_build, ctx->stream));
  return PECC_OK;
}

pecc_status pecc_solve_host(pecc_ctx *ctx, const double *R_host, uint64_t seed, double *xy_host,
                            int32_t *iters_host, int32_t *status_host, uint8_t *feasible_host,
                            double *max_overlap_host) {
  if (!ctx || (ctx->num > 0 && !R_host)) return PECC_ERR_ARG;
  if (ctx->num == 0) return PECC_OK;
  // inputs: the radii go up, the layout is drawn on the device
  double *dR = (double *)ctx->stage;                     // [num] doubles
  uint8_t *dfeas = (uint8_t *)(ctx->stage + 8 * (size_t)ctx->num);   // [num]
  double *dmo = (double *)(ctx->stage + 16 * (size_t)ctx->num);      // [num]
  int32_t *dit = (int32_t *)(ctx->stage + 24 * (size_t)ctx->num);    // [num]
  int32_t *dst = dit + ctx->num;                                      // [num]
  CK(cudaMemcpyAsync(dR, R_host, sizeof(double) * ctx->num, cudaMemcpyHostToDevice, ctx->stream));
  const bool same = ctx->radius_set && ctx->radius_host_known &&
                    std::memcmp(ctx->radius_host.data(), R_host, sizeof(double) * ctx->num) == 0;
  pecc_status s;
  if (!same) {
    if ((s = pecc_set_radius(ctx, dR))) return s;
    ctx->radius_host.assign(R_host, R_host + ctx->num);
    ctx->radius_host_known = true;
  }
  if ((s = pecc_init_random(ctx, seed))) return s;
  if ((s = pecc_descend(ctx, nullptr, nullptr))) return s;
  if ((s = pecc_check_feasible(ctx, ctx->cfg.feas_tol, dfeas, dmo))) return s;
  CK(launch_outputs(ctx->out, ctx->num, dit, dst, nullptr, nullptr, nullptr, nullptr, ctx->stream));
  if (xy_host) {
    double *dxy = (double *)ctx->xo;  // 2 * total doubles
    if ((s = pecc_get_positions(ctx, dxy))) return s;
    CK(cudaMemcpyAsync(xy_host, dxy, sizeof(double) * 2 * ctx->total, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (iters_host) CK(cudaMemcpyAsync(iters_host, dit, sizeof(int32_t) * ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  if (status_host) CK(cudaMemcpyAsync(status_host, dst, sizeof(int32_t) * ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  if (feasible_host) CK(cudaMemcpyAsync(feasible_host, dfeas, ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  if (max_overlap_host) CK(cudaMemcpyAsync(max_overlap_host, dmo, sizeof(double) * ctx->num, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PECC_OK;
}


}  // extern "C"

// ------------------------------------------------------------------ SED (Sec. 5.2)
struct pecc_sed {
  pecc_ctx *cand = nullptr;  // the candidate slots: instance q's slot j is descent instance q*M + j
  pecc_sed_config sc{};
  int num = 0, M = 0;
  std::vector<int32_t> n;
  std::vector<double> R;
  int64_t total = 0;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  SedParams p{};
  bool radius_set = false, started = false;
  std::string err;
};

static pecc_status sfail(pecc_sed *s, pecc_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  else g_create_err = buf;
  return st;
}

#define SCK(call)                                                                               \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return sfail(sed, PECC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T> static pecc_status salloc(pecc_sed *sed, T **p, size_t count) {
  void *v = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e != cudaSuccess) return sfail(sed, PECC_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  sed->allocs.push_back(v);
  *p = (T *)v;
  return PECC_OK;
}

extern "C" {

void pecc_sed_config_default(pecc_sed_config *c) {
  std::memset(c, 0, sizeof *c);
  c->max_candidates = 25;
  c->s_iter = 500;
  c->e_feas = 1e-25;
  c->amp = 0.8;
  c->shared_r = 0;
  c->check_every = 8;
}

pecc_status pecc_sed_destroy(pecc_sed *sed) {
  if (!sed) return PECC_OK;
  cudaStreamSynchronize(sed->stream);
  if (sed->cand) pecc_destroy(sed->cand);
  for (void *v : sed->allocs) cudaFree(v);
  delete sed;
  return PECC_OK;
}

pecc_status pecc_sed_create(const pecc_config *cfg, const pecc_sed_config *sc, void *stream, pecc_sed **out) {
  if (!out) return sfail(nullptr, PECC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || !sc) return sfail(nullptr, PECC_ERR_ARG, "cfg or sed config is NULL");
  if (sc->max_candidates < 1 || sc->max_candidates > 64)
    return sfail(nullptr, PECC_ERR_ARG, "max_candidates must be in 1..64");
  if (sc->s_iter < 0 || sc->check_every < 1) return sfail(nullptr, PECC_ERR_ARG, "s_iter >= 0 and check_every >= 1");
  if (!(sc->amp >= 0.0) || !std::isfinite(sc->amp) || !(sc->e_feas >= 0.0))
    return sfail(nullptr, PECC_ERR_ARG, "amp finite and >= 0, e_feas >= 0");
  if (cfg->num_instances < 0 || (cfg->num_instances > 0 && !cfg->n))
    return sfail(nullptr, PECC_ERR_ARG, "num_instances < 0 or n is NULL");
  const int num = cfg->num_instances, M = sc->max_candidates;
  if ((int64_t)num * M > (int64_t)1 << 30) return sfail(nullptr, PECC_ERR_ARG, "too many candidate slots");
  for (int q = 0; q < num; ++q)
    if (cfg->n[q] < 0 || cfg->n[q] >= kGridMinN)
      return sfail(nullptr, PECC_ERR_ARG, "n[%d] must be in 0..%d (one block per candidate)", q, kGridMinN - 1);
  pecc_sed *sed = new pecc_sed();
  sed->sc = *sc;
  sed->num = num;
  sed->M = M;
  sed->n.assign(cfg->n, cfg->n + num);
  sed->stream = (cudaStream_t)stream;
  for (int v : sed->n) sed->total += v;
  auto bail = [&](pecc_status st) {
    g_create_err = sed->err;
    pecc_sed_destroy(sed);
    return st;
  };
  std::vector<int32_t> cn((size_t)num * M);
  for (int q = 0; q < num; ++q)
    for (int j = 0; j < M; ++j) cn[(size_t)q * M + j] = sed->n[q];
  pecc_config c2 = *cfg;
  c2.num_instances = num * M;
  c2.n = cn.data();
  pecc_status st = pecc_create(&c2, stream, &sed->cand);
  if (st) return bail(sfail(sed, st, "candidate context: %s", g_create_err.c_str()));
  pecc_ctx *ctx = sed->cand;
  SedParams &p = sed->p;
  p.num = num;
  p.M = M;
  p.init_mode = cfg->init_mode;
  p.shared_r = sc->shared_r ? 1 : 0;
  p.from32 = cfg->precision == PECC_FP32 ? 1 : 0;
  p.amp = sc->amp;
  p.e_feas = sc->e_feas;
  int32_t *nd = nullptr;
  int64_t *off = nullptr;
  double *Rd = nullptr;
  if ((st = salloc(sed, &nd, num)) || (st = salloc(sed, &off, num + 1)) || (st = salloc(sed, &Rd, num)) ||
      (st = salloc(sed, &p.x, sed->total)) || (st = salloc(sed, &p.xb, sed->total)) ||
      (st = salloc(sed, &p.Ex, num)) || (st = salloc(sed, &p.Eb, num)) || (st = salloc(sed, &p.m, num)) ||
      (st = salloc(sed, &p.sel, num)) || (st = salloc(sed, &p.done, num)) || (st = salloc(sed, &p.iters, num)) ||
      (st = salloc(sed, &p.porder, num)) || (st = salloc(sed, &p.scan, num)) ||
      (st = salloc(sed, &p.list, (size_t)num * M)) || (st = salloc(sed, &p.count, 1)) || (st = salloc(sed, &p.left, 1)) ||
      (st = salloc(sed, &p.active, 1)))
    return bail(st);
  p.n = nd;
  p.off = off;
  p.R = Rd;
  std::vector<int64_t> oh(num + 1, 0);
  for (int q = 0; q < num; ++q) oh[q + 1] = oh[q] + sed->n[q];
  std::vector<int32_t> po(num);
  std::iota(po.begin(), po.end(), 0);
  std::stable_sort(po.begin(), po.end(), [&](int a, int b) { return sed->n[a] > sed->n[b]; });
  cudaStream_t s = sed->stream;
  SCK(cudaMemcpyAsync(nd, sed->n.data(), sizeof(int32_t) * std::max(num, 0), cudaMemcpyHostToDevice, s));
  SCK(cudaMemcpyAsync(off, oh.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, s));
  SCK(cudaMemcpyAsync(p.porder, po.data(), sizeof(int32_t) * std::max(num, 0), cudaMemcpyHostToDevice, s));
  SCK(cudaMemsetAsync(p.iters, 0, sizeof(int32_t) * std::max(num, 1), s));
  SCK(cudaMemsetAsync(p.done, 0, sizeof(int32_t) * std::max(num, 1), s));
  SCK(cudaStreamSynchronize(s));
  p.cdesc = ctx->desc;
  p.cout = ctx->out;
  p.c64 = ctx->x64;
  p.c32 = ctx->x32;
  // the descent processes the active slots the list step writes into its order array
  p.list = ctx->order;
  ctx->num_dev = p.count;
  *out = sed;
  return PECC_OK;
}

const char *pecc_sed_last_error(pecc_sed *sed) { return sed ? sed->err.c_str() : g_create_err.c_str(); }

pecc_ctx *pecc_sed_context(pecc_sed *sed) { return sed ? sed->cand : nullptr; }

pecc_status pecc_sed_set_radius(pecc_sed *sed, const double *R_dev) {
  if (!sed) return PECC_ERR_ARG;
  if (sed->num == 0) { sed->radius_set = true; return PECC_OK; }
  if (!R_dev) return sfail(sed, PECC_ERR_ARG, "R_dev is NULL");
  sed->R.resize(sed->num);
  SCK(cudaMemcpyAsync(sed->R.data(), R_dev, sizeof(double) * sed->num, cudaMemcpyDeviceToHost, sed->stream));
  SCK(cudaStreamSynchronize(sed->stream));
  std::vector<double> R2((size_t)sed->num * sed->M);
  for (int q = 0; q < sed->num; ++q)
    for (int j = 0; j < sed->M; ++j) R2[(size_t)q * sed->M + j] = sed->R[q];
  double *tmp = nullptr;
  SCK(cudaMalloc(&tmp, sizeof(double) * R2.size()));
  cudaError_t e = cudaMemcpyAsync(tmp, R2.data(), sizeof(double) * R2.size(), cudaMemcpyHostToDevice, sed->stream);
  pecc_status st = e ? PECC_ERR_CUDA : pecc_set_radius(sed->cand, tmp);
  cudaStreamSynchronize(sed->stream);
  cudaFree(tmp);
  if (e) return sfail(sed, PECC_ERR_CUDA, "upload radii: %s", cudaGetErrorString(e));
  if (st) return sfail(sed, st, "%s", pecc_last_error(sed->cand));
  SCK(cudaMemcpyAsync((double *)sed->p.R, R_dev, sizeof(double) * sed->num, cudaMemcpyDeviceToDevice, sed->stream));
  sed->radius_set = true;
  return PECC_OK;
}

static pecc_status sed_descend(pecc_sed *sed) {
  pecc_status st = pecc_descend(sed->cand, nullptr, nullptr);
  return st ? sfail(sed, st, "%s", pecc_last_error(sed->cand)) : PECC_OK;
}

pecc_status pecc_sed_start(pecc_sed *sed, uint64_t seed) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->radius_set) return sfail(sed, PECC_ERR_ARG, "pecc_sed_set_radius has not been called");
  sed->p.seed = seed;
  sed->p.it = 0;
  sed->started = true;
  if (sed->num == 0) return PECC_OK;
  SCK(cudaMemsetAsync(sed->p.iters, 0, sizeof(int32_t) * sed->num, sed->stream));
  SCK(launch_sed_init(sed->p, sed->stream));
  SCK(launch_sed_prepare(sed->p, 1, sed->stream));
  pecc_status st = sed_descend(sed);
  if (st) return st;
  SCK(launch_sed_select(sed->p, nullptr, 1, sed->stream));
  return PECC_OK;
}

pecc_status pecc_sed_set_state(pecc_sed *sed, const double *x_dev, const double *Ex_dev, uint64_t seed, int32_t it) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->radius_set) return sfail(sed, PECC_ERR_ARG, "pecc_sed_set_radius has not been called");
  if (it < 0) return sfail(sed, PECC_ERR_ARG, "it must be >= 0");
  sed->p.seed = seed;
  sed->p.it = it;
  sed->started = true;
  if (sed->num == 0) return PECC_OK;
  if (!x_dev || !Ex_dev) return sfail(sed, PECC_ERR_ARG, "NULL state");
  const size_t xb = sizeof(double2) * (size_t)sed->total;
  SCK(cudaMemcpyAsync(sed->p.x, x_dev, xb, cudaMemcpyDeviceToDevice, sed->stream));
  SCK(cudaMemcpyAsync(sed->p.xb, x_dev, xb, cudaMemcpyDeviceToDevice, sed->stream));
  SCK(cudaMemcpyAsync(sed->p.Ex, Ex_dev, sizeof(double) * sed->num, cudaMemcpyDeviceToDevice, sed->stream));
  SCK(cudaMemcpyAsync(sed->p.Eb, Ex_dev, sizeof(double) * sed->num, cudaMemcpyDeviceToDevice, sed->stream));
  SCK(cudaMemsetAsync(sed->p.iters, 0, sizeof(int32_t) * sed->num, sed->stream));
  SCK(cudaMemsetAsync(sed->p.done, 0, sizeof(int32_t) * sed->num, sed->stream));
  return PECC_OK;
}

pecc_status pecc_sed_prepare(pecc_sed *sed) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->started) return sfail(sed, PECC_ERR_ARG, "pecc_sed_start or pecc_sed_set_state first");
  SCK(launch_sed_prepare(sed->p, 0, sed->stream));
  return PECC_OK;
}

pecc_status pecc_sed_descend(pecc_sed *sed) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->started) return sfail(sed, PECC_ERR_ARG, "pecc_sed_start or pecc_sed_set_state first");
  return sed->num ? sed_descend(sed) : PECC_OK;
}

pecc_status pecc_sed_select(pecc_sed *sed, const double *E_cand_dev) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->started) return sfail(sed, PECC_ERR_ARG, "pecc_sed_start or pecc_sed_set_state first");
  SCK(launch_sed_select(sed->p, E_cand_dev, 0, sed->stream));
  sed->p.it += 1;
  return PECC_OK;
}

pecc_status pecc_sed_get(pecc_sed *sed, double *x_dev, double *xbest_dev, double *Ex_dev, double *Eb_dev,
                         int32_t *iters_dev, int32_t *status_dev, int32_t *m_dev, int32_t *sel_dev, double *cand_dev) {
  if (!sed) return PECC_ERR_ARG;
  if (sed->num == 0) return PECC_OK;
  cudaStream_t s = sed->stream;
  const size_t xb = sizeof(double2) * (size_t)sed->total, eb = sizeof(double) * sed->num, ib = sizeof(int32_t) * sed->num;
  if (x_dev) SCK(cudaMemcpyAsync(x_dev, sed->p.x, xb, cudaMemcpyDeviceToDevice, s));
  if (xbest_dev) SCK(cudaMemcpyAsync(xbest_dev, sed->p.xb, xb, cudaMemcpyDeviceToDevice, s));
  if (Ex_dev) SCK(cudaMemcpyAsync(Ex_dev, sed->p.Ex, eb, cudaMemcpyDeviceToDevice, s));
  if (Eb_dev) SCK(cudaMemcpyAsync(Eb_dev, sed->p.Eb, eb, cudaMemcpyDeviceToDevice, s));
  if (iters_dev) SCK(cudaMemcpyAsync(iters_dev, sed->p.iters, ib, cudaMemcpyDeviceToDevice, s));
  if (m_dev) SCK(cudaMemcpyAsync(m_dev, sed->p.m, ib, cudaMemcpyDeviceToDevice, s));
  if (sel_dev) SCK(cudaMemcpyAsync(sel_dev, sed->p.sel, ib, cudaMemcpyDeviceToDevice, s));
  if (status_dev) SCK(launch_sed_status(sed->p, status_dev, s));
  if (cand_dev) {
    pecc_status st = pecc_get_positions(sed->cand, cand_dev);
    if (st) return sfail(sed, st, "%s", pecc_last_error(sed->cand));
  }
  return PECC_OK;
}

pecc_status pecc_sed_iterate(pecc_sed *sed, int32_t max_iterations, int32_t *ran_host, int32_t *left_host) {
  if (!sed) return PECC_ERR_ARG;
  if (!sed->started) return sfail(sed, PECC_ERR_ARG, "pecc_sed_start or pecc_sed_set_state first");
  if (max_iterations < 0) return sfail(sed, PECC_ERR_ARG, "max_iterations must be >= 0");
  int ran = 0;
  int32_t left = 0;
  if (sed->num > 0) {
    // the instances not done yet: the list step counts those with candidates (the prepared
    // candidates are drawn again, identically, by the first iteration below)
    SCK(launch_sed_prepare(sed->p, 0, sed->stream));
    SCK(cudaMemcpyAsync(&left, sed->p.active, sizeof(int32_t), cudaMemcpyDeviceToHost, sed->stream));
    SCK(cudaStreamSynchronize(sed->stream));
  }
  while (left > 0 && ran < max_iterations && sed->p.it < sed->sc.s_iter) {
    SCK(launch_sed_prepare(sed->p, 0, sed->stream));
    pecc_status st = sed_descend(sed);
    if (st) return st;
    SCK(launch_sed_select(sed->p, nullptr, 0, sed->stream));
    sed->p.it += 1;
    ++ran;
    if (ran % sed->sc.check_every == 0) {
      SCK(cudaMemcpyAsync(&left, sed->p.left, sizeof(int32_t), cudaMemcpyDeviceToHost, sed->stream));
      SCK(cudaStreamSynchronize(sed->stream));
    }
  }
  if (ran > 0) {
    SCK(cudaMemcpyAsync(&left, sed->p.left, sizeof(int32_t), cudaMemcpyDeviceToHost, sed->stream));
    SCK(cudaStreamSynchronize(sed->stream));
  }
  if (ran_host) *ran_host = ran;
  if (left_host) *left_host = left;
  return PECC_OK;
}


pecc_status pecc_frame_run(pecc_sed *sed, pecc_ctx *adj, const double *Rb_dev, uint64_t seed, int32_t outer,
                           int32_t sed_iters, double lambda0, int32_t rounds, double *Rbest_dev, double *xbest_dev,
                           double *Rtrace_dev, int32_t *adj_stats_dev) {
  if (!sed || !adj) return PECC_ERR_ARG;
  if (!Rb_dev || !Rbest_dev || !xbest_dev) return sfail(sed, PECC_ERR_ARG, "pecc_frame_run: NULL pointer");
  if (outer < 0 || sed_iters < 0 || rounds < 0 || !(lambda0 >= 0.0) || !std::isfinite(lambda0))
    return sfail(sed, PECC_ERR_ARG, "pecc_frame_run: outer, sed_iters, rounds >= 0 and lambda0 finite, >= 0");
  if (adj->num != sed->num || adj->n != sed->n)
    return sfail(sed, PECC_ERR_ARG, "pecc_frame_run: the adjustment context must hold the search's instances");
  if (adj->stream != sed->stream)
    return sfail(sed, PECC_ERR_ARG, "pecc_frame_run: the search and the adjustment context must share a stream");
  const int num = sed->num;
  if (num == 0) return PECC_OK;
  cudaStream_t s = sed->stream;
  double *R = nullptr, *Rn = nullptr;
  double2 *x = nullptr;
  int32_t *iters = nullptr, *status = nullptr, *stats = nullptr;
  pecc_status st = PECC_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    cudaFree(R); cudaFree(Rn); cudaFree(x); cudaFree(iters); cudaFree(status); cudaFree(stats);
  };
  if (cudaMalloc(&R, sizeof(double) * num) || cudaMalloc(&Rn, sizeof(double) * num) ||
      cudaMalloc(&x, sizeof(double2) * std::max<int64_t>(sed->total, 1)) ||
      cudaMalloc(&iters, sizeof(int32_t) * num) || cudaMalloc(&status, sizeof(int32_t) * num) ||
      cudaMalloc(&stats, sizeof(int32_t) * 2 * num)) {
    cleanup();
    return sfail(sed, PECC_ERR_OOM, "pecc_frame_run: scratch allocation failed");
  }
  auto ctx_err = [&](pecc_status e) { return sfail(sed, e, "%s", pecc_last_error(adj)); };
  auto adjust = [&](const double *Rin, double *Rout, const double2 *xin) -> pecc_status {
    pecc_status e;
    if ((e = pecc_set_radius(adj, Rin))) return ctx_err(e);
    if ((e = pecc_set_positions(adj, (const double *)xin))) return ctx_err(e);
    if (cudaMemcpyAsync(Rout, Rin, sizeof(double) * num, cudaMemcpyDeviceToDevice, s)) return PECC_ERR_CUDA;
    if ((e = pecc_adjust_container(adj, Rout, lambda0, rounds, iters, status, stats))) return ctx_err(e);
    if ((e = pecc_get_positions(adj, (double *)x))) return ctx_err(e);
    if (adj_stats_dev &&
        (launch_add_i32(num, iters, adj_stats_dev, s) || launch_add_i32(2 * num, stats, adj_stats_dev + num, s)))
      return PECC_ERR_CUDA;
    return PECC_OK;
  };
  if (adj_stats_dev && cudaMemsetAsync(adj_stats_dev, 0, sizeof(int32_t) * 3 * num, s)) {
    cleanup();
    return sfail(sed, PECC_ERR_CUDA, "pecc_frame_run: clearing the statistics");
  }
  do {
    // x* = GBO(random_solution(n, R_b)); (x*, R*) = adjust(x*, R_b)
    if ((st = pecc_sed_set_radius(sed, Rb_dev)) || (st = pecc_sed_start(sed, seed))) break;
    if ((st = pecc_sed_get(sed, (double *)x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr)))
      break;
    if ((st = adjust(Rb_dev, Rbest_dev, x))) break;
    if (cudaMemcpyAsync(xbest_dev, x, sizeof(double2) * sed->total, cudaMemcpyDeviceToDevice, s) ||
        (Rtrace_dev && cudaMemcpyAsync(Rtrace_dev, Rbest_dev, sizeof(double) * num, cudaMemcpyDeviceToDevice, s))) {
      st = PECC_ERR_CUDA;
      break;
    }
    for (int t = 0; t < outer && st == PECC_OK; ++t) {
      // R = min(R_b, R*); x = SED(n, R); (x, R) = adjust(x, R); keep it when R < R*
      if (launch_frame_radius(num, Rb_dev, Rbest_dev, R, s)) { st = PECC_ERR_CUDA; break; }
      int32_t ran = 0, left = 0;
      if ((st = pecc_sed_set_radius(sed, R)) || (st = pecc_sed_start(sed, seed + 1 + (uint64_t)t)) ||
          (st = pecc_sed_iterate(sed, sed_iters, &ran, &left)))
        break;
      if ((st = pecc_sed_get(sed, nullptr, (double *)x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                             nullptr)))
        break;
      if ((st = adjust(R, Rn, x))) break;
      if (launch_frame_record(sed->p, Rn, x, Rbest_dev, (double2 *)xbest_dev, s) ||
          (Rtrace_dev && cudaMemcpyAsync(Rtrace_dev + (size_t)(t + 1) * num, Rbest_dev, sizeof(double) * num,
                                         cudaMemcpyDeviceToDevice, s))) {
        st = PECC_ERR_CUDA;
        break;
      }
    }
  } while (false);
  cleanup();
  if (st == PECC_ERR_CUDA && sed->err.empty()) sfail(sed, st, "pecc_frame_run: CUDA error");
  return st;
}

}  // extern "C"
