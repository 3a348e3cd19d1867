/*
 * pecc.h -- C ABI of the GB300 descent library for the elastic model of
 * packing equal circles in a circle (arXiv 2303.02650).
 *
 * The library evaluates and minimises the overlap energy of Sec. 3.2
 *
 *   d_ij = max(0, 2 - |c_i - c_j|)           (Eq. 3, pair overlap depth)
 *   d_i0 = max(0, |c_i| + 1 - R)             (Eq. 3, container overlap depth)
 *   E(x) = sum_{i<j} d_ij^2 + sum_i d_i0^2   (Eq. 5)
 *
 * over neighbor lists Gamma(i) = {j != i : l_ij < l_cut} (Sec. 4.3) that are
 * rebuilt adaptively (Algorithm ANM, Sec. 4.3, plus a Verlet displacement
 * rule), by geometric batch optimisation (Algorithm GBO, Sec. 4.1): circles
 * are split into k sector batches and each batch takes quasi-Newton steps
 * (Eq. 8, with the inverse Hessian of Eq. 10 / Eq. 11 kept as m secant pairs)
 * in Gauss-Seidel order.
 *
 * Conventions for every call:
 *  - A context holds num_instances independent instances; instance q has n[q]
 *    unit circles in a container of radius R[q] centred at the origin.
 *  - Positions are interleaved (x, y) pairs, instances concatenated in n[]
 *    order: circle i of instance q is at element 2 * (off[q] + i), where
 *    off[q] = n[0] + ... + n[q-1].
 *  - Pointers named *_dev are DEVICE pointers owned by the caller (for
 *    example a torch CUDA tensor's data_ptr()); *_host are host pointers.
 *  - Every call is ordered on the context's CUDA stream and returns after
 *    enqueueing, except those that read something back and so synchronise the
 *    stream: pecc_neighbor_count,
 *    pecc_export_neighbors, pecc_autotune, pecc_phase_times, pecc_solve_host,
 *    pecc_destroy; pecc_sed_create, pecc_sed_set_radius, pecc_sed_iterate (every
 *    check_every iterations), pecc_sed_destroy, pecc_frame_run, pecc_mlp_destroy.
 *  - Argument errors are returned synchronously.  Errors found on the device
 *    (non-finite coordinates, a neighbor list over capacity, a time budget
 *    exceeded) are written to the per-instance status outputs of the call
 *    that found them; nothing aborts, traps or spins without a bound.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef PECC_H
#define PECC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pecc_ctx pecc_ctx;

typedef enum {
    PECC_OK = 0,
    PECC_ERR_ARG = 1,          /* invalid argument (message in pecc_last_error) */
    PECC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    PECC_ERR_OOM = 3,          /* device allocation failed */
    PECC_ERR_NBR_OVERFLOW = 4, /* a neighbor list exceeded its capacity */
    PECC_ERR_NONFINITE = 5,    /* NaN or Inf coordinates or energy */
    PECC_ERR_TIMEOUT = 6       /* the time budget ran out */
} pecc_status;

/* Per-instance outcome of pecc_descend (status_dev values). */
enum {
    PECC_DESC_CONVERGED = 0,   /* E <= e_tol */
    PECC_DESC_STATIONARY = 1,  /* sum over batches of |g_p|_2 <= gsum_tol (Algorithm GBO) */
    PECC_DESC_STALLED = 2,     /* no batch could lower its energy in a sweep */
    PECC_DESC_MAX_ITER = 3,    /* max_iter sweeps done */
    PECC_DESC_NBR_OVERFLOW = 4,
    PECC_DESC_NONFINITE = 5,
    PECC_DESC_TIMEOUT = 6
};

/* Arithmetic of the context. */
enum {
    PECC_FP64 = 0,          /* plain FP64 everywhere */
    PECC_FP32 = 1,          /* FP32 coordinates, energy, gradient and accumulation */
    PECC_FP32_POLISH64 = 2  /* FP32 bulk descent, then an FP64 polish descent */
};

/* Partitions of Sec. 4.1: the three geometric ones, and the random one (a uniform Philox-keyed
 * order of the circles, cut into the same contiguous batch sizes). */
enum { PECC_PART_SECTOR = 0, PECC_PART_ANNULUS = 1, PECC_PART_FENCE = 2, PECC_PART_RANDOM = 3 };

/* Initial layout of Sec. 5.1. */
enum { PECC_INIT_DISK = 0, PECC_INIT_SQUARE = 1 };

typedef struct {
    int32_t num_instances;
    const int32_t *n;       /* host array [num_instances], each n >= 0; copied at create */
    int32_t precision;      /* PECC_FP64 | PECC_FP32 | PECC_FP32_POLISH64 */
    double l_cut;           /* neighbor cutoff; 2.5 (the paper uses 4), must exceed 2 */
    double rebuild_disp;    /* Verlet half-skin: a rebuild happens before a batch step when
                               2 * max displacement since the last build + step_max exceeds
                               2 * rebuild_disp; 0.25 = (l_cut - 2) / 2 */
    double step_max;        /* cap on any circle's move in one batch step; 0.1 */
    int32_t lbfgs_m;        /* secant pairs kept per batch, 1..10; 10 */
    int32_t max_iter;       /* sweeps of the main descent; 2000 */
    int32_t polish_max_iter;/* sweeps of the FP64 polish (PECC_FP32_POLISH64); 1000 */
    int32_t k_batches;      /* batches per instance; 0 = 1 (n < 300), 3 (n < 500), 5 */
    int32_t partition;      /* PECC_PART_*; sector */
    int32_t max_trials;     /* backtracking trials per line search; 30 */
    int32_t anm;            /* 1: ANM deferred rebuilds on (Algorithm ANM); 1 */
    int32_t init_mode;      /* PECC_INIT_*; disk of radius R - 1 */
    double e_tol;           /* stop when E <= e_tol; 1e-20 */
    double gsum_tol;        /* stop when sum_p |g_p|_2 <= gsum_tol; 1e-12 */
    double c1;              /* Armijo constant; 1e-4 */
    double curv_eps;        /* keep a pair only if s'y > curv_eps |s| |y|; 1e-10 */
    double polish_gate;     /* polish only instances whose FP32 energy is <= this; 1e-4 */
    double feas_tol;        /* feasible when the largest overlap depth <= feas_tol; 1e-9 */
    double nbr_capacity;    /* neighbor entries reserved per circle; 16 */
    int64_t time_budget_ns; /* per pecc_descend call, measured on the device; 0 = none */
    int32_t block_threads;  /* threads per instance block; 0 = about two circles per thread
                               (at most 256 when instances outnumber SMs), or pecc_autotune's */
    int32_t blocks_per_sm;  /* target of resident instance blocks per SM, which also caps each
                               block's shared-memory share of the working set; 0 = 2 when
                               instances outnumber SMs, else 1, or pecc_autotune's */
    double stall_rel;       /* FP32 phase of PECC_FP32_POLISH64 / PECC_FP32 ends (status STALLED) when
                               E fell by less than stall_rel (relative) over stall_window sweeps:
                               binary32 has reached its resolution; 1e-3 */
    int32_t stall_window;   /* sweeps per stagnation check of the FP32 phase; 10 (0 = off) */
    int32_t polish_k;       /* batches of the FP64 polish (at most k_batches); 1 (0 = k_batches) */
    int32_t smem_per_block; /* bytes of dynamic shared memory per instance block at most (the rest
                               of the working set stays in global memory and the SM's L1 keeps the
                               room); 0 = the block's whole share of the SM */
    double polish_stall_rel;      /* the FP64 polish ends (status STALLED) when E fell by less than
                                     polish_stall_rel (relative) over polish_stall_window sweeps: a
                                     polish that stagnates above zero energy is at a jammed local
                                     minimum; 1e-2 */
    int32_t polish_stall_window;  /* sweeps per stagnation check of the polish; 100 (0 = off) */
    int32_t fuse_phases;    /* PECC_FP32_POLISH64: 1 = each instance's FP32 descent and polish run
                               back to back in one block of one kernel (long polishes overlap other
                               instances' descents; pecc_phase_times then reports the fused kernel
                               as the first phase and 0 for the polish), 0 = two kernels; 1 */
    uint64_t partition_seed;  /* PECC_PART_RANDOM: the Philox key; circle i of instance q draws
                                 counter (i, 0, q, 3 * 2^30); 0 */
    int32_t qn_dense;       /* 1: each batch keeps its inverse Hessian H_p explicitly and updates
                               it by Eq. 11 (the paper's BFGS; H_p starts as I and is rescaled to
                               (s'y / y'y) I before its first update), in place of the m secant
                               pairs.  Needs PECC_FP64 and instances below 16384 circles; the
                               first pecc_descend allocates sum over batches of (2 |B_p|)^2
                               doubles (32 MB for n = 1000, k = 1).  lbfgs_m is then unused; 0 */
    double list_outer;      /* the descent (instances below 16384 circles) keeps an outer list of
                               the pairs closer than l_cut + list_outer, built from the cell grid,
                               and makes every list of Sec. 4.3 (each ANM and Verlet rebuild) by
                               filtering it, as long as twice the largest displacement since the
                               outer list's build stays below list_outer (else the outer list is
                               rebuilt first).  The filter applies the same predicate to the same
                               coordinates, so the lists are the same set as a build from the cell
                               grid; only their order within a row can differ.  0 = every rebuild
                               from the cell grid, else in [2^-9, 64]; 0.5 */
} pecc_config;

/* Fill *cfg with the defaults listed above (num_instances = 0, n = NULL). */
void pecc_config_default(pecc_config *cfg);

/* Create a context on the current CUDA device for num_instances independent problems of the kind
 * Sec. 3.1 states: instance q places n[q] unit circles in a container of radius R[q] so that no
 * two overlap (Eq. 1) and none leaves the container (Eq. 2).  The radii come later
 * (pecc_set_radius).  stream: a cudaStream_t (NULL = the legacy default stream).  Allocates every
 * device buffer the context needs (sized from n[] and the config); *out receives the context or
 * NULL.  Synchronous (device allocations and uploads). */
pecc_status pecc_create(const pecc_config *cfg, void *stream, pecc_ctx **out);

/* Synchronise the stream and free the context and its device memory. */
pecc_status pecc_destroy(pecc_ctx *ctx);

/* Container radii R of the problem statement (Sec. 3.1; the container constraint of Eq. 2 and the
 * wall depth of Eq. 3 use them): R_dev = device double[num_instances], each R finite and > 0.
 * Stream-ordered and asynchronous: a kernel copies the radii and sizes each instance's cell grid
 * on the device (the cell tables were allocated at pecc_create for the largest grid an instance
 * can get, max(16, ceil(2 sqrt(n))) cells per side), so R_dev must stay valid until the stream
 * has run the call.  A radius that is not finite and > 0 is not an argument error (it is not read
 * on the host): its instance gets R = NaN, and its energies, descents (status
 * PECC_DESC_NONFINITE) and feasibility checks (max_overlap NaN) say so. */
pecc_status pecc_set_radius(pecc_ctx *ctx, const double *R_dev);

/* Coordinates: xy_dev = device double[2 * sum n].  FP32 contexts round them to binary32. */
pecc_status pecc_set_positions(pecc_ctx *ctx, const double *xy_dev);

/* Random initial layout of Sec. 5.1 on the device (init_mode of the config): circle i of
 * instance q uses Philox4x32-10 with key (seed lo, seed hi) and counter (i, attempt, q, 0);
 * two 53-bit uniforms give a candidate in [-(R-1), R-1]^2, accepted inside the disk. */
pecc_status pecc_init_random(pecc_ctx *ctx, uint64_t seed);

/* Current coordinates as doubles: xy_dev = device double[2 * sum n].  For
 * PECC_FP32_POLISH64 these are the polished FP64 coordinates after pecc_descend. */
pecc_status pecc_get_positions(pecc_ctx *ctx, double *xy_dev);

/* (Re)build the neighbor lists Gamma of every instance (Sec. 4.3) by cell binning and a
 * key sort.  force = 0 rebuilds only instances whose largest displacement since their
 * last build exceeds rebuild_disp; rebuilt_dev (device int32[num_instances], may be NULL)
 * receives 1 where a list was rebuilt. */
pecc_status pecc_rebuild_neighbors(pecc_ctx *ctx, int32_t force, int32_t *rebuilt_dev);

/* Number of stored neighbor entries (sum over instances of sum_i |Gamma(i)|); synchronises.
 * PECC_ERR_NBR_OVERFLOW when an instance's last build exceeded its capacity (nbr_capacity). */
pecc_status pecc_neighbor_count(pecc_ctx *ctx, int64_t *nnz_host);

/* Export the neighbor lists as one CSR over all circles: row_ptr_dev = device
 * int32[sum n + 1], col_dev = device int32[cap] of global circle indices, each row
 * ascending.  PECC_ERR_ARG if cap is below the count of pecc_neighbor_count, and its
 * PECC_ERR_NBR_OVERFLOW after an overflowed build.  Synchronises. */
pecc_status pecc_export_neighbors(pecc_ctx *ctx, int32_t *row_ptr_dev, int32_t *col_dev, int64_t cap);

/* Export the cell binning of the last build: key_dev = device uint32[sum n] (cell index
 * cy * ncx + cx with cell side l_cut (1 + 2^-20)), order_dev = device int32[sum n], the
 * circles of each instance stably sorted by key (local indices). */
pecc_status pecc_export_cells(pecc_ctx *ctx, uint32_t *key_dev, int32_t *order_dev);

/* Coordinates of an instance the energy + gradient call stages in shared memory at most
 * (PECC_ENERGY_STAGE_BYTES / 8 circles in FP32, / 16 in FP64 and the mixed arithmetic). */
#define PECC_ENERGY_STAGE_BYTES (96 * 1024)

/* Energy (Eq. 5, neighbor-list form of Sec. 4.3) and gradient of every instance at the
 * current coordinates over the current lists: E_dev = device double[num_instances];
 * grad_dev = device float2[sum n] (FP32 contexts) or double2[sum n] (PECC_FP64).
 * One block per instance with its coordinates staged in shared memory (one launch for all
 * instances up to PECC_ENERGY_STAGE_BYTES of coordinates); larger instances take one thread
 * per circle and a per-instance reduction.
 * The gradient is gathered (no atomics) and E is summed in a fixed order (deterministic).
 * An instance whose last build overflowed its list capacity (nbr_capacity) gets E = NaN and
 * a NaN gradient. */
pecc_status pecc_energy_grad(pecc_ctx *ctx, double *E_dev, void *grad_dev);

/* Same, with an explicit arithmetic: eval = PECC_FP64 (double2 gradient), PECC_FP32
 * (float2) or PECC_FP32_POLISH64 (the mixed arithmetic of the polish: FP64 coordinates,
 * pair differences and 4 - l^2, FP32 elsewhere; float2 gradient).  The lists must have
 * been built in the matching precision (FP32 for PECC_FP32, FP64 otherwise):
 * pecc_rebuild_neighbors_ex. */
pecc_status pecc_energy_grad_ex(pecc_ctx *ctx, int32_t eval, double *E_dev, void *grad_dev);
pecc_status pecc_rebuild_neighbors_ex(pecc_ctx *ctx, int32_t eval, int32_t force, int32_t *rebuilt_dev);

/* Descend every instance from its current coordinates (Algorithm GBO with ANM, Sec. 4.1 /
 * Sec. 4.3) as one persistent, graph-captured launch: one thread block per instance, a
 * device work queue over instances (largest first).  PECC_FP32_POLISH64 runs the FP32
 * descent and then the FP64 polish on instances whose FP32 energy is <= polish_gate.
 * iters_dev (device int32[num_instances], may be NULL): sweeps done (both phases);
 * status_dev (device int32[num_instances], may be NULL): PECC_DESC_* of the last phase. */
pecc_status pecc_descend(pecc_ctx *ctx, int32_t *iters_dev, int32_t *status_dev);

/* Parity hook for tests of the descent's own neighbor lists (Sec. 4.3): every following
 * pecc_descend writes, for each instance below 16384 circles, the lists in force at the end of its
 * first phase (the binary32 lists of the FP32 descent of PECC_FP32 and PECC_FP32_POLISH64, the
 * binary64 lists of PECC_FP64) and the coordinates they were built at.
 *   stride   entries kept per row, >= 1
 *   cnt_dev  device int32[sum n]: the row length of circle i (caller's numbering), or -1 when the
 *            row is longer than stride or the phase ended without a complete build
 *   col_dev  device int32[sum n * stride]: row i at i * stride, instance-local circle indices, in
 *            the descent's own order (not sorted)
 *   xb_dev   device double[2 * sum n]: the coordinates of that build (binary32 values widened in
 *            the FP32 phase)
 * cnt_dev = NULL turns the hook off.  The buffers must outlive every descent that writes them.
 * Changing the hook makes the next pecc_descend capture its graph again.  Asynchronous. */
pecc_status pecc_set_list_dump(pecc_ctx *ctx, int32_t stride, int32_t *cnt_dev, int32_t *col_dev, double *xb_dev);

/* Per-instance energies after the last pecc_descend: device double[num_instances]. */
pecc_status pecc_get_energy(pecc_ctx *ctx, double *E_dev);

/* Feasibility (Eq. 1, Eq. 2): largest pair overlap depth over ALL pairs (a fresh FP64 cell
 * list with cutoff l_cut > 2 holds every overlapping pair) and largest container overlap
 * depth, in FP64 with correctly rounded operations; feasible_dev (device uint8[num]) is 1
 * where the larger of the two is <= tol, max_overlap_dev (device double[num]) receives it.
 * An instance that cannot be checked (a non-finite coordinate, or more list entries than twice
 * its capacity) gets max_overlap NaN and feasible 0. */
pecc_status pecc_check_feasible(pecc_ctx *ctx, double tol, uint8_t *feasible_dev, double *max_overlap_dev);

/* The whole path from host memory: copy R_host (double[num]) to the device, draw the
 * initial layout from seed, descend, check feasibility with feas_tol, and copy back
 * xy_host (double[2 sum n], may be NULL), iters_host / status_host (int32[num], may be
 * NULL), feasible_host (uint8[num], may be NULL) and max_overlap_host (double[num], may
 * be NULL).  Synchronises. */
pecc_status pecc_solve_host(pecc_ctx *ctx, const double *R_host, uint64_t seed, double *xy_host,
                            int32_t *iters_host, int32_t *status_host, uint8_t *feasible_host,
                            double *max_overlap_host);

/* Counters of the last pecc_descend, device int32[num_instances] each (may be NULL):
 * neighbor builds, builds that changed Gamma, line-search trials. */
pecc_status pecc_get_counters(pecc_ctx *ctx, int32_t *builds_dev, int32_t *changes_dev, int32_t *trials_dev);

/* Per-instance statistics of the last pecc_descend: stats_dev = device int32[num_instances][10]:
 * iters (both phases), status, neighbor builds, builds that changed Gamma, line-search trials,
 * memory resets, stalled batch steps, polished (0/1), sweeps of the first phase, trials of the
 * first phase. */
pecc_status pecc_get_stats(pecc_ctx *ctx, int32_t *stats_dev);

/* Device time of the kernels of the last pecc_descend, from events recorded on the context's
 * stream inside the descent graph: ms_host[0] = first phase (FP64 or FP32 descent kernel),
 * ms_host[1] = FP64 polish kernel (0 when there is none), ms_host[2] = the whole descent.
 * Synchronises on the last event. */
pecc_status pecc_phase_times(pecc_ctx *ctx, float *ms_host);

/* Autotuner of the descent's launch shape: for threads per instance block in {128, 256, 512} and
 * a target of {1, 2, 4, 5, 6} blocks per SM (which sets the shared-memory share of the working set
 * and the compiled kernel instance: the largest register budget that reaches the target), it
 * draws a layout from seed and times `sweeps` sweeps of the context's own instances, and keeps the
 * shape with the most circle-sweeps per second for the following pecc_descend calls (also after
 * pecc_set_radius, which only re-sizes the shared-memory share).  The FP64 polish of
 * PECC_FP32_POLISH64 runs with min(block, 256) threads and the same target.  The caller's
 * coordinates are restored.  Synchronises; allocates a temporary copy of the coordinates.
 * block_out / bps_out (host, may be NULL) receive the chosen threads per block and target. */
pecc_status pecc_autotune(pecc_ctx *ctx, int32_t sweeps, uint64_t seed, int32_t *block_out, int32_t *bps_out);

/* The launch shape the context uses for its descent kernels. */
pecc_status pecc_get_launch(pecc_ctx *ctx, int32_t *block_threads, int32_t *blocks_per_sm, int32_t *grid);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start.  Not in the paper: a per-circle MLP (25 -> 128 -> 128 -> 128 -> 2, ReLU,
 * BF16 weights on the fifth-generation tensor cores (tcgen05.mma, accumulators in TMEM, tiles of
 * 128 rows), FP32 accumulation and FP32 master weights) maps the local
 * neighborhood of a circle to a displacement; it is trained on displacements the descent itself
 * makes, and the plain descent stays its fallback and the test of its moves (a warm-start move of
 * an instance is kept only if it does not raise that instance's energy).
 * Features of circle i (FP32, correctly rounded): frame e_r = c_i/|c_i| (e_r = (1, 0) at the
 * origin), e_t = (-e_r.y, e_r.x); the 12 nearest other centres within 4.5 (by squared distance,
 * then index) as offsets c_j - c_i in (e_r, e_t) coordinates, zero-padded: 24 values; then
 * min(R - |c_i| - 1, 4.5).  Row layout float[25].
 * Parameters: float[pecc_mlp_num_params()] = W1[128][25] b1[128] W2[128][128] b2[128]
 * W3[128][128] b3[128] W4[2][128] b4[2]; the network reads BF16 copies of the weights and rounds
 * every GEMM input (features, activations, back-propagated gradients) to BF16.
 * --------------------------------------------------------------------------------------------- */
typedef struct pecc_mlp pecc_mlp;

/* Number of MLP parameters (36610). */
int32_t pecc_mlp_num_params(void);

/* Create a network with He-uniform weights from Philox4x32-10 (key = seed) and zero biases; all
 * its calls run on stream (a cudaStream_t; NULL = legacy default stream). */
pecc_status pecc_mlp_create(uint64_t seed, void *stream, pecc_mlp **out);
pecc_status pecc_mlp_destroy(pecc_mlp *mlp);

/* Copy the FP32 parameters to / from device memory (float[num_params]); set refreshes the BF16
 * copies and does not touch the Adam moments. */
pecc_status pecc_mlp_get_params(pecc_mlp *mlp, float *params_dev);
pecc_status pecc_mlp_set_params(pecc_mlp *mlp, const float *params_dev);

/* Forward: feat_dev float[rows][25] -> out_dev float[rows][2] (displacement in the circle's frame). */
pecc_status pecc_mlp_forward(pecc_mlp *mlp, const float *feat_dev, int64_t rows, float *out_dev);

/* Gradient of the loss L = (1/rows) sum_r |out_r - target_r|^2 with respect to the FP32 parameters
 * (grad_dev float[num_params]); loss_dev (float[1], may be NULL) receives L. */
pecc_status pecc_mlp_grad(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                          float *grad_dev, float *loss_dev);

/* The same two calls writing what the tensor cores computed, for tests against a CPU restatement:
 * forward: trace_dev float[rows][3][128], the bf16 activations of the three hidden layers (as
 * floats); grad: fwd_trace_dev the same for the forward pass of the gradient, bwd_trace_dev
 * float[rows][4][128], the bf16 back-propagated dZ3, dZ2, dZ1 (ReLU-masked, as floats), then in the
 * fourth row the bf16 output gradient dO (2 values) and the outputs (2 values). */
pecc_status pecc_mlp_forward_trace(pecc_mlp *mlp, const float *feat_dev, int64_t rows, float *out_dev,
                                   float *trace_dev);
pecc_status pecc_mlp_grad_trace(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                                float *grad_dev, float *loss_dev, float *fwd_trace_dev, float *bwd_trace_dev);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on L with learning rate lr. */
pecc_status pecc_mlp_train_step(pecc_mlp *mlp, const float *feat_dev, const float *target_dev, int64_t rows,
                                float lr, float *loss_dev);

/* Features of every circle of an FP32 context at its current coordinates: float[sum n][25]. */
pecc_status pecc_features(pecc_ctx *ctx, const float *unused, float *feat_dev);

/* Training targets: each circle's displacement from xbefore_dev (double[2 sum n]) to the current
 * FP32 coordinates, in the frame of its position in xbefore: float[sum n][2]. */
pecc_status pecc_targets(pecc_ctx *ctx, const double *xbefore_dev, float *target_dev);

/* Warm start of an FP32 context: rounds x (features -> network -> move each circle by the
 * proposal, clipped to 0.25, in the global frame); a round's move of an instance is kept only if
 * its neighbor-list energy (Eq. 5) does not rise, else the instance is put back.  accepted_dev
 * (int32[num_instances], may be NULL) is increased by the number of rounds kept. */
pecc_status pecc_warm_start(pecc_ctx *ctx, pecc_mlp *mlp, int32_t rounds, int32_t *accepted_dev);

/* The same with the largest move of a circle per round as a parameter (max_move > 0; the call
 * above uses 0.25).  The moves need no bound for the check that follows them (the energy after a
 * round is evaluated over lists rebuilt at the moved layout); the bound limits the damage of a
 * poor proposal. */
pecc_status pecc_warm_start_ex(pecc_ctx *ctx, pecc_mlp *mlp, int32_t rounds, double max_move, int32_t *accepted_dev);

/* Largest instance pecc_check_feasible_noalloc accepts. */
#define PECC_NOALLOC_MAX_N 4096

/* The feasibility check of pecc_check_feasible for ONE instance, without any device allocation.
 * The paper has no counterpart: this is a service for callers that cannot call cudaMalloc
 * (code running while its stream is captured into a CUDA graph, plug-ins whose host owns all
 * device memory, real-time loops).  Its scratch (about 0.85 MB) is a fixed array in device
 * memory that every GPU loading the library holds until the process exits.
 *   xy_dev          device double[2 n], interleaved (x, y)
 *   n               0 .. PECC_NOALLOC_MAX_N circles, else PECC_ERR_ARG (nothing launched)
 *   R, l_cut        container radius > 0, neighbor cutoff > 2 of the FP64 cell list
 *   tol             feasible when the largest depth <= tol
 *   feasible_dev    device uint8[1];  max_overlap_dev  device double[1] (NaN if not checkable)
 *   stream          cudaStream_t the kernel is enqueued on (NULL = legacy default stream)
 * The first call on a device takes the array's device address (cudaGetSymbolAddress, with that
 * device current) and keeps it for the life of the process; make that first call before any
 * stream capture.  A cudaDeviceReset (or a lost context) on that device leaves the kept address
 * stale: make no further call on that device afterwards.  Every call shares the one array and
 * finds the previous call's contents there (the kernel clears what must start at zero); calls
 * whose kernels overlap on the GPU race on it, so order them on one stream.  Errors are returned
 * synchronously; the message is in pecc_last_error(NULL).  The neighbor list holds at most
 * 2 (16 n + 64) entries, as pecc_check_feasible's in a context with the default nbr_capacity of
 * 16: with that context the results are identical for the same coordinates, NaN included (an
 * instance whose list would exceed it gets max_overlap NaN and feasible 0). */
pecc_status pecc_check_feasible_noalloc(const double *xy_dev, int32_t n, double R, double l_cut, double tol,
                                        uint8_t *feasible_dev, double *max_overlap_dev, void *stream);

/* Container adjustment (Sec. 4.2, Algorithm adjust_container, Eq. 12): with z = (x, R) and
 * U(z, lambda) = E(x, R) + lambda R^2, for each of `rounds` rounds a limited-memory BFGS (the
 * descent's step, one batch, lbfgs_m pairs, a fresh memory each round) minimises U over all of z,
 * then lambda is halved; the paper's schedule is lambda0 = 1e-4, rounds = 35.  A round ends when
 * |grad U| <= gsum_tol, when no step is accepted, or after max_iter iterations.
 * Arithmetic: PECC_FP64 contexts run it in binary64.  The others use the polish arithmetic for
 * the pair terms (binary64 differences and 4 - l^2, binary32 depths and forces), binary32
 * gradients and quasi-Newton vectors, and binary64 energies and radius.  There, while E is
 * large (a large lambda), a round settles within about 1e-6 of U's minimum; the schedule's late
 * rounds (E -> 0) settle the radius as binary64 does. */
/* Arguments:
 *   R_dev       device double[num_instances]: the starting radii in, the adjusted radii out (the
 *               context's own radii, those of pecc_set_radius, are left as they are)
 *   iters_dev   device int32[num_instances]: quasi-Newton iterations over all rounds
 *   status_dev  device int32[num_instances]: status of the last round (1 stationary, 2 stalled,
 *               3 max_iter; 4: list capacity exceeded, or an instance of 16384 circles or more,
 *               which this call does not adjust; 0 for an empty instance)
 *   stats_dev   device int32[num_instances][2] or NULL: line-search trials (energy + gradient
 *               evaluations) and stored pairs visited by the two-loop recursion, over all rounds
 * Starts from the context's coordinates (those of the last descent, pecc_set_positions or
 * pecc_init_random) and replaces them with the adjusted layout.  Stream-ordered, asynchronous;
 * the first call allocates the binary64 secant pairs (lbfgs_m <= 10 slots per circle).
 * Errors: PECC_ERR_ARG for NULL pointers, rounds < 0, lambda0 < 0 or not finite, lbfgs_m > 10. */
pecc_status pecc_adjust_container(pecc_ctx *ctx, double *R_dev, double lambda0, int32_t rounds, int32_t *iters_dev,
                                  int32_t *status_dev, int32_t *stats_dev);

/* Self-test of the bounded wait of the grid barrier that the whole-GPU descent of large instances
 * uses (the wait is measured on %globaltimer; past its limit the waiting block raises an error
 * flag that every block sees, and the descent ends with status 6).  Four blocks wait at a barrier
 * that expects a fifth, so no arrival releases it; every wait must end by itself after
 * timeout_ns.  Runs on the current device and the legacy default stream; synchronises.
 *   timeout_ns        the wait limit to test (> 0, at most 10 s)
 *   failed_host       host int32[1]: 1 when the barrier reported the failed wait, else 0
 *   waited_ns_host    host int64[1]: how long block 0 waited
 * Returns PECC_ERR_ARG for a bad argument, PECC_ERR_CUDA (message in pecc_last_error(NULL)) if
 * the launch or a copy failed. */
pecc_status pecc_selftest_grid_barrier(int64_t timeout_ns, int32_t *failed_host, int64_t *waited_ns_host);

/* Text of the last error on this context (or of the last failed pecc_create when ctx is NULL). */
const char *pecc_last_error(pecc_ctx *ctx);

/* ====================================================================================== SED
 * The solution-space exploring and descent heuristic (Sec. 5.2, Algorithm SED) over a batch of
 * instances at fixed container radii.
 *   Start:     x_q <- GBO(random_solution(n_q, R_q)); x*_q <- x_q.
 *   Iteration: unless E(x*_q) <= e_feas, instance q perturbs x_q into
 *              m_q = max(1, J(E(x_q))) candidates, with J(E) = ceil(-log10 E) and m_q capped at
 *              max_candidates.  Each candidate moves every circle by r ~ U(-amp, amp) in x and
 *              in y.  Each candidate is descended by GBO, then x_q <- select(U) (Eq. 18): the
 *              least candidate energy if it is below E(x_q), otherwise a draw with probabilities
 *              softmax(J(y)).  Finally x*_q <- x_q when E(x_q) < E(x*_q).
 * All the candidates of all instances descend together: the object owns a descent context with
 * max_candidates slots per instance.  Each iteration runs on the device without waiting for the
 * host.  The random numbers are Philox4x32-10 keyed by the seed:
 *   - initial layout of instance q: counter (i, attempt, q, 0), as pecc_init_random;
 *   - candidate j of iteration it: counter (i, it, q, 2^31 + j) for circle i;
 *   - select draw: counter (0, it, q, 2^30), u = 53 bits of the first two words in [0, 1).
 * Energies E are the descent's (pecc_get_energy) in the context's arithmetic; x and x* are
 * binary64.  Instances must have fewer than 16384 circles (one block per candidate). */
typedef struct pecc_sed pecc_sed;

typedef struct {
  int32_t max_candidates; /* candidate slots per instance, 1..64 (25: every J while E > 1e-25) */
  int32_t s_iter;         /* SED iterations at most (the paper: 500) */
  double e_feas;          /* stop an instance once E(x*) <= e_feas (the paper: 1e-25) */
  double amp;             /* perturbation half-width (the paper: 0.8) */
  int32_t shared_r;       /* 1: one r for both coordinates of a circle (the formula as printed);
                             0: independent draws for x and y (default) */
  int32_t check_every;    /* pecc_sed_iterate reads the count of running instances every this
                             many iterations (one host synchronisation each) */
} pecc_sed_config;

/* Defaults: 25 candidates, 500 iterations, e_feas 1e-25, amp 0.8, independent draws, check 8. */
void pecc_sed_config_default(pecc_sed_config *c);

/* cfg: the instances (num_instances, n) and the descent's settings, used for every candidate
 * (e_tol is GBO's own energy stop: set it to e_feas to descend candidates as far as SED asks).
 * stream: cudaStream_t or NULL.  Errors: PECC_ERR_ARG (bad configuration, n >= 16384),
 * PECC_ERR_OOM; the message is in pecc_sed_last_error(NULL). */
pecc_status pecc_sed_create(const pecc_config *cfg, const pecc_sed_config *sc, void *stream, pecc_sed **out);
pecc_status pecc_sed_destroy(pecc_sed *sed);
const char *pecc_sed_last_error(pecc_sed *sed);

/* R_dev: device double[num_instances], finite and > 0.  Synchronises the stream. */
pecc_status pecc_sed_set_radius(pecc_sed *sed, const double *R_dev);

/* Lines 1-3 of Algorithm SED for every instance: random layouts (cfg.init_mode), their GBO, and
 * x = x* = the result.  Resets the iteration counter to 0.  Asynchronous. */
pecc_status pecc_sed_start(pecc_sed *sed, uint64_t seed);

/* Replaces the start: x = x* = x_dev (device double[2 * sum n], interleaved), E(x) = E(x*) =
 * Ex_dev (device double[num_instances]), iteration counter it, random numbers keyed by seed. */
pecc_status pecc_sed_set_state(pecc_sed *sed, const double *x_dev, const double *Ex_dev, uint64_t seed, int32_t it);

/* Up to max_iterations SED iterations, each stopping instances whose E(x*) <= e_feas, and never
 * past s_iter in all.  Stops early once no instance is running.  The stream is synchronised every
 * check_every iterations and at the end.  ran_host: iterations run; left_host: instances still
 * running (either may be NULL). */
pecc_status pecc_sed_iterate(pecc_sed *sed, int32_t max_iterations, int32_t *ran_host, int32_t *left_host);

/* The three steps of one iteration, for tests and custom drivers:
 *   prepare: m_q and the candidates;
 *   descend: GBO of the active candidates;
 *   select:  Eq. 18 and the record.  E_cand_dev is device double[num_instances * max_candidates]
 *            (slot q * max_candidates + j) replacing the descent's energies, or NULL.
 * select advances the iteration counter.  All asynchronous. */
pecc_status pecc_sed_prepare(pecc_sed *sed);
pecc_status pecc_sed_descend(pecc_sed *sed);
pecc_status pecc_sed_select(pecc_sed *sed, const double *E_cand_dev);

/* Read the state (device pointers; any may be NULL):
 *   x_dev, xbest_dev  double[2 * sum n]    x and x*
 *   Ex_dev, Eb_dev    double[num]          E(x) and E(x*)
 *   iters_dev         int32[num]           SED iterations each instance ran
 *   status_dev        int32[num]           0 once E(x*) <= e_feas, else 3
 *   m_dev, sel_dev    int32[num]           the last iteration's candidate count (0: done before
 *                                          it) and selected candidate
 * cand_dev: double[2 * max_candidates * sum n]: the candidate slots, instance by instance (slot j
 * of instance q at 2 * (max_candidates * off_q + j * n_q)), or NULL. */
pecc_status pecc_sed_get(pecc_sed *sed, double *x_dev, double *xbest_dev, double *Ex_dev, double *Eb_dev,
                         int32_t *iters_dev, int32_t *status_dev, int32_t *m_dev, int32_t *sel_dev, double *cand_dev);

/* The candidate descent context (owned by sed: do not destroy it, nor change its radii or
 * positions), for pecc_get_stats, pecc_phase_times, pecc_get_launch and pecc_get_energy of the
 * last descent (slot q * max_candidates + j; slots not active in that descent keep older values).
 * NULL if sed is NULL. */
pecc_ctx *pecc_sed_context(pecc_sed *sed);

/* ============================================================================ the framework
 * The framework of Sec. 5.1 (Algorithm 5) over a batch, with `outer` iterations in place of the
 * cut-off time:
 *   x* = GBO(random_solution(n, R_b)); (x*, R*) = adjust_container(x*, R_b);
 *   repeat outer times: R = min(R_b, R*); x = SED(n, R) (sed_iters iterations);
 *                       (x, R) = adjust_container(x, R); x*, R* = x, R where R < R*.
 *   sed        the search (its instances, candidate slots and descent settings); the first layout
 *              draws under `seed` (pecc_sed_start), SED call t under seed + 1 + t
 *   adj        a context holding the same instances on the same stream, for the container
 *              adjustments (its arithmetic and iteration limits apply); its radii and positions
 *              are overwritten
 *   Rb_dev     device double[num_instances]: the best-known radii R_b
 *   Rbest_dev  device double[num_instances] out: R*;  xbest_dev device double[2 * sum n] out: x*
 *   Rtrace_dev device double[(outer + 1) * num_instances] or NULL: R* after the first adjustment
 *              and after every iteration (row t + 1 after iteration t)
 *   adj_stats_dev device int32[3 * num_instances] or NULL: summed over every adjustment of the
 *              call, the iterations (first num), then per instance {line-search trials, pairs
 *              visited by the two-loop recursion} (as pecc_adjust_container's stats)
 * Synchronises (radius changes); allocates scratch for the call.  Errors: PECC_ERR_ARG for NULL
 * outputs, negative counts, or an adjustment context with other instances; the message is in
 * pecc_sed_last_error(sed). */
pecc_status pecc_frame_run(pecc_sed *sed, pecc_ctx *adj, const double *Rb_dev, uint64_t seed, int32_t outer,
                           int32_t sed_iters, double lambda0, int32_t rounds, double *Rbest_dev, double *xbest_dev,
                           double *Rtrace_dev, int32_t *adj_stats_dev);

#ifdef __cplusplus
}
#endif

#endif /* PECC_H */
