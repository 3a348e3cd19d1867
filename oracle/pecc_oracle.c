/*
 * pecc_oracle.c -- plain, slow FP64 CPU oracle for the elastic-model descent of
 * "Geometric Batch Optimization for the Packing Equal Circles in a Circle
 * Problem on Large Scale" (arXiv 2303.02650).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, call or
 * execute this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Compile with -O2 -ffp-contract=off (no FMA contraction): every floating
 * point operation below is then a single correctly rounded IEEE operation in
 * the written order, so the integer decisions taken from floating point
 * (cell keys, neighbor predicates, sector order) are reproducible bit for bit.
 *
 * What each function follows:
 *   init            Sec. 5.1 (random_solution of the framework algorithm),
 *                   read as uniform in the disk of radius R-1; the paper's
 *                   square U(-R,R)^2 is mode 1.  Random numbers come from
 *                   Philox4x32-10 (Salmon et al., SC'11), implemented here
 *                   from its published definition.
 *   neighbors       Sec. 4.3, the neighbor set Gamma(i) = {j != i : l_ij < l_cut}.
 *   energy          Def. "Overlapping distance" (Eq. 3) and "Elastic energy"
 *                   (Eq. 5); batch energy Eq. 7 and its neighbor-list form
 *                   (Sec. 4.3).
 *   gradient        derived from Eq. 3 / Eq. 5 (the paper does not print it).
 *   partition       Sec. 4.1 sector / annulus / fence partitions, batch sizes
 *                   floor(n/k) or ceil(n/k).
 *   descent         Algorithm "GBO" (Sec. 4.1): per-batch quasi-Newton steps
 *                   Eq. 8 with the inverse-Hessian action of Eq. 10 / Eq. 11
 *                   taken in limited-memory form (m pairs), step length from
 *                   a backtracking (Armijo) search in place of the argmin of
 *                   Eq. 9, Gauss-Seidel order over batches, ANM after every
 *                   sweep (Algorithm "ANM", Sec. 4.3), and the stop test on
 *                   the sum of batch gradient norms.
 *   dense BFGS      Eq. 10 / Eq. 11 applied as written, used by the tests to
 *                   pin the limited-memory two-loop recursion.
 *   feasibility     Eq. 1 / Eq. 2: maximum pair and boundary overlap depth.
 *   adjustment      Sec. 4.2, Eq. 12 (container adjustment by L-BFGS over (x, R)).
 *   SED             Sec. 5.2, Algorithm SED and the select operator of Eq. 18.
 *   framework       Sec. 5.1, the framework algorithm (GBO, adjustment, then SED and
 *                   adjustment repeated at min(R_b, R*), keeping the smallest feasible radius).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, key      */
/* bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53 random bits from two words -> double in [0, 1). */
static double u53(uint32_t hi, uint32_t lo)
{
    uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Random initial layout of one instance (Sec. 5.1).
 * mode 0: uniform in the disk of radius R-1 by rejection from the square
 *         [-(R-1), R-1]^2; attempt a of circle i draws counter (i, a, inst, 0).
 * mode 1: the paper's square, x, y ~ U(-R, R), counter (i, 0, inst, 0).
 * xy receives interleaved (x, y) doubles.
 */
void orc_init_positions(int n, double R, uint64_t seed, int inst, int mode, double *xy)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double rr = R - 1.0;
    for (int i = 0; i < n; i++) {
        double x = 0.0, y = 0.0;
        if (mode == 1) {
            uint32_t ctr[4] = {(uint32_t)i, 0u, (uint32_t)inst, 0u}, w[4];
            orc_philox4x32_10(ctr, key, w);
            x = R * (2.0 * u53(w[0], w[1]) - 1.0);
            y = R * (2.0 * u53(w[2], w[3]) - 1.0);
        } else if (rr > 0.0) {
            for (uint32_t a = 0; a < 64u; a++) {
                uint32_t ctr[4] = {(uint32_t)i, a, (uint32_t)inst, 0u}, w[4];
                orc_philox4x32_10(ctr, key, w);
                double cx = rr * (2.0 * u53(w[0], w[1]) - 1.0);
                double cy = rr * (2.0 * u53(w[2], w[3]) - 1.0);
                if (cx * cx + cy * cy <= rr * rr) {
                    x = cx;
                    y = cy;
                    break;
                }
            }
        }
        xy[2 * i] = x;
        xy[2 * i + 1] = y;
    }
}

/* ------------------------------------------------------------------------ */
/* Cell binning.  Cell side cs = l_cut * (1 + 2^-20): a hair above the cutoff */
/* so that rounding in (x + R) / cs can never put two circles closer than     */
/* l_cut two cells apart.  Coordinates are clamped into the grid (clamping is */
/* monotone, so it never separates a neighbor pair by more than one cell).    */
/* A sparse instance gets at most max(16, ceil(2 sqrt n)) cells per side (the */
/* side then grows to 2R / ncx), so cell storage stays O(n).                  */
/* ------------------------------------------------------------------------ */
void orc_cell_grid(double R, double l_cut, int n, double *inv_cs, int *ncx)
{
    double cs = l_cut * (1.0 + 1.0 / 1048576.0);
    double inv = 1.0 / cs;
    double w = ceil((2.0 * R) * inv);
    int cap = (int)ceil(2.0 * sqrt((double)n));
    if (cap < 16) cap = 16;
    int nc = (w >= 1.0) ? (w > 65535.0 ? 65535 : (int)w) : 1;
    if (nc > cap) {
        nc = cap;
        inv = (double)nc / (2.0 * R);
    }
    *inv_cs = inv;
    *ncx = nc;
}

static int cell_coord(double v, double R, double inv, int nc)
{
    double f = (v + R) * inv;
    if (!(f >= 0.0)) return 0; /* negative or NaN */
    if (f >= (double)nc) return nc - 1;
    return (int)f;
}

void orc_cell_keys(int n, const double *xy, double R, double l_cut, uint32_t *key)
{
    double inv;
    int nc;
    orc_cell_grid(R, l_cut, n, &inv, &nc);
    for (int i = 0; i < n; i++) {
        int cx = cell_coord(xy[2 * i], R, inv, nc);
        int cy = cell_coord(xy[2 * i + 1], R, inv, nc);
        key[i] = (uint32_t)cy * (uint32_t)nc + (uint32_t)cx;
    }
}

/* Stable counting sort of circle indices by key: order[] and cell_start[ncell+1]. */
void orc_cell_sort(int n, const uint32_t *key, int ncell, int32_t *order, int32_t *cell_start)
{
    for (int c = 0; c <= ncell; c++) cell_start[c] = 0;
    for (int i = 0; i < n; i++) cell_start[key[i] + 1]++;
    for (int c = 0; c < ncell; c++) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell > 0 ? ncell : 1));
    for (int c = 0; c < ncell; c++) fill[c] = cell_start[c];
    for (int i = 0; i < n; i++) order[fill[key[i]]++] = i;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Neighbor predicate of Sec. 4.3: j in Gamma(i) iff j != i and               */
/* dx*dx + dy*dy < l_cut^2, every operation correctly rounded, no FMA.        */
/* prec32 != 0 evaluates it in binary32 on coordinates that are binary32      */
/* values (the precision the FP32 path stores), else in binary64.             */
/* ------------------------------------------------------------------------ */
static int nbr_pred(const double *xy, int i, int j, double lc2, int prec32)
{
    if (prec32) {
        float dx = (float)xy[2 * i] - (float)xy[2 * j];
        float dy = (float)xy[2 * i + 1] - (float)xy[2 * j + 1];
        float s = dx * dx;
        float t = dy * dy;
        s = s + t;
        return s < (float)lc2;
    }
    double dx = xy[2 * i] - xy[2 * j];
    double dy = xy[2 * i + 1] - xy[2 * j + 1];
    double s = dx * dx;
    double t = dy * dy;
    s = s + t;
    return s < lc2;
}

/* All-pairs neighbor lists (rows ascending).  Returns nnz, or -nnz_needed if cap is too small. */
int64_t orc_neighbors_brute(int n, const double *xy, double l_cut, int prec32,
                            int32_t *row_ptr, int32_t *col, int64_t cap)
{
    double lc2 = l_cut * l_cut;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            if (j == i || !nbr_pred(xy, i, j, lc2, prec32)) continue;
            if (nnz < cap) col[nnz] = j;
            nnz++;
        }
        row_ptr[i + 1] = (int32_t)(nnz < cap ? nnz : cap);
    }
    return nnz <= cap ? nnz : -nnz;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Cell-list neighbor lists over the 3x3 block of cells, rows sorted ascending. */
int64_t orc_neighbors_cells(int n, const double *xy, double R, double l_cut, int prec32,
                            int32_t *row_ptr, int32_t *col, int64_t cap)
{
    double inv;
    int nc;
    orc_cell_grid(R, l_cut, n, &inv, &nc);
    int ncell = nc * nc;
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(n, xy, R, l_cut, key);
    orc_cell_sort(n, key, ncell, order, start);
    double lc2 = l_cut * l_cut;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int i = 0; i < n; i++) {
        int cx = (int)(key[i] % (uint32_t)nc), cy = (int)(key[i] / (uint32_t)nc);
        int len = 0;
        for (int by = cy - 1; by <= cy + 1; by++) {
            if (by < 0 || by >= nc) continue;
            for (int bx = cx - 1; bx <= cx + 1; bx++) {
                if (bx < 0 || bx >= nc) continue;
                int c = by * nc + bx;
                for (int t = start[c]; t < start[c + 1]; t++) {
                    int j = order[t];
                    if (j != i && nbr_pred(xy, i, j, lc2, prec32)) row[len++] = j;
                }
            }
        }
        qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int t = 0; t < len; t++) {
            if (nnz < cap) col[nnz] = row[t];
            nnz++;
        }
        row_ptr[i + 1] = (int32_t)(nnz < cap ? nnz : cap);
    }
    free(key);
    free(order);
    free(start);
    free(row);
    return nnz <= cap ? nnz : -nnz;
}

/* ------------------------------------------------------------------------ */
/* Energy (Eq. 3, Eq. 5) and its gradient.                                   */
/* Energies are summed with Neumaier compensation so that the oracle is the  */
/* more accurate side of every comparison.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s, c;
} ksum;

static void ks_add(ksum *k, double v)
{
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v))
        k->c += (k->s - t) + v;
    else
        k->c += (v - t) + k->s;
    k->s = t;
}

static double ks_get(const ksum *k) { return k->s + k->c; }

/* d_i0 of Eq. 3 (second part). */
static double bound_depth(double x, double y, double R, double *r_out)
{
    double r = sqrt(x * x + y * y);
    if (r_out) *r_out = r;
    double d = r + 1.0 - R;
    return d > 0.0 ? d : 0.0;
}

/* Eq. 5 over all pairs i < j, plus the boundary terms. */
double orc_energy_allpairs(int n, const double *xy, double R)
{
    ksum e = {0.0, 0.0};
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            double l = sqrt(dx * dx + dy * dy);
            double d = 2.0 - l;
            if (d > 0.0) ks_add(&e, d * d);
        }
        double b = bound_depth(xy[2 * i], xy[2 * i + 1], R, NULL);
        if (b > 0.0) ks_add(&e, b * b);
    }
    return ks_get(&e);
}

/*
 * Gradient of circle i over its neighbor row (every j in Gamma(i)):
 *   dE/dx_i = sum_j -2 d_ij (x_i - x_j) / l_ij  +  2 d_i0 x_i / |c_i|.
 * A coincident pair (l_ij = 0) or a centred circle (|c_i| = 0) contributes 0,
 * a valid subgradient at those kinks; *degen counts such pairs.
 */
static void grad_row(int i, const double *xy, double R, const int32_t *row_ptr, const int32_t *col,
                     double *gx, double *gy, int *degen)
{
    double xi = xy[2 * i], yi = xy[2 * i + 1];
    double ax = 0.0, ay = 0.0;
    for (int t = row_ptr[i]; t < row_ptr[i + 1]; t++) {
        int j = col[t];
        double dx = xi - xy[2 * j], dy = yi - xy[2 * j + 1];
        double l = sqrt(dx * dx + dy * dy);
        double d = 2.0 - l;
        if (d > 0.0) {
            if (l > 0.0) {
                double c = -2.0 * d / l;
                ax += c * dx;
                ay += c * dy;
            } else if (degen) {
                (*degen)++;
            }
        }
    }
    double r;
    double b = bound_depth(xi, yi, R, &r);
    if (b > 0.0 && r > 0.0) {
        double c = 2.0 * b / r;
        ax += c * xi;
        ay += c * yi;
    }
    *gx = ax;
    *gy = ay;
}

/* Neighbor-list energy (each unordered pair once, from the row of the larger index). */
double orc_energy_csr(int n, const double *xy, double R, const int32_t *row_ptr, const int32_t *col)
{
    ksum e = {0.0, 0.0};
    for (int i = 0; i < n; i++) {
        for (int t = row_ptr[i]; t < row_ptr[i + 1]; t++) {
            int j = col[t];
            if (j >= i) continue;
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            double l = sqrt(dx * dx + dy * dy);
            double d = 2.0 - l;
            if (d > 0.0) ks_add(&e, d * d);
        }
        double b = bound_depth(xy[2 * i], xy[2 * i + 1], R, NULL);
        if (b > 0.0) ks_add(&e, b * b);
    }
    return ks_get(&e);
}

/* Energy and full gradient over the neighbor lists; returns E, writes g[2n]. */
double orc_energy_grad_csr(int n, const double *xy, double R, const int32_t *row_ptr,
                           const int32_t *col, double *g, int *degen)
{
    for (int i = 0; i < n; i++) grad_row(i, xy, R, row_ptr, col, &g[2 * i], &g[2 * i + 1], degen);
    return orc_energy_csr(n, xy, R, row_ptr, col);
}

/* All-pairs gradient (brute force reference for the tests). */
void orc_grad_allpairs(int n, const double *xy, double R, double *g)
{
    for (int i = 0; i < n; i++) {
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            double l = sqrt(dx * dx + dy * dy);
            double d = 2.0 - l;
            if (d > 0.0 && l > 0.0) {
                double c = -2.0 * d / l;
                ax += c * dx;
                ay += c * dy;
            }
        }
        double r;
        double b = bound_depth(xy[2 * i], xy[2 * i + 1], R, &r);
        if (b > 0.0 && r > 0.0) {
            ax += 2.0 * b / r * xy[2 * i];
            ay += 2.0 * b / r * xy[2 * i + 1];
        }
        g[2 * i] = ax;
        g[2 * i + 1] = ay;
    }
}

/*
 * Batch energy of Eq. 7 in its neighbor-list form (Sec. 4.3):
 *   E(x_p) = sum_{i in B_p} sum_{j in Gamma(i)} d_ij^2 [j not in B_p or j < i]
 *            + sum_{i in B_p} d_i0^2
 * (the garbled boundary subscript of the printed neighbor form is read as
 * i in B_p).  members[0..nb) lists B_p; batch_of[j] gives each circle's batch.
 */
double orc_batch_energy(const double *xy, double R, const int32_t *row_ptr, const int32_t *col,
                        const int32_t *members, int nb, const int32_t *batch_of, int p)
{
    ksum e = {0.0, 0.0};
    for (int a = 0; a < nb; a++) {
        int i = members[a];
        for (int t = row_ptr[i]; t < row_ptr[i + 1]; t++) {
            int j = col[t];
            if (batch_of[j] == p && j >= i) continue;
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            double l = sqrt(dx * dx + dy * dy);
            double d = 2.0 - l;
            if (d > 0.0) ks_add(&e, d * d);
        }
        double b = bound_depth(xy[2 * i], xy[2 * i + 1], R, NULL);
        if (b > 0.0) ks_add(&e, b * b);
    }
    return ks_get(&e);
}

/* Gradient of E(x_p) with respect to x_p: the full gradient restricted to B_p. */
static void batch_grad(const double *xy, double R, const int32_t *row_ptr, const int32_t *col,
                       const int32_t *members, int nb, double *g)
{
    for (int a = 0; a < nb; a++)
        grad_row(members[a], xy, R, row_ptr, col, &g[2 * a], &g[2 * a + 1], NULL);
}

/* ------------------------------------------------------------------------ */
/* Geometric partitions (Sec. 4.1).                                           */
/* Sector key: the pseudo-angle, strictly increasing in the polar angle on    */
/* [0, 2 pi) (the printed arctan(y/x) is read as the full polar angle):       */
/*   y >= 0: 1 - x / (|x| + |y|),  y < 0: 3 + x / (|x| + |y|),  origin: 0.    */
/* Annulus key: sqrt(x^2 + y^2).  Fence key: x.                               */
/* Random (mode 3): "partition all circles into k sets randomly" is read as a */
/* uniformly random order cut into the same contiguous sizes; circle i's key  */
/* is 53 bits of Philox4x32-10 counter (i, 0, inst, 3 * 2^30) under the      */
/* partition seed (the order by (key, index) is a uniform permutation).       */
/* Stable by (key, index); the first n mod k batches hold ceil(n/k) circles.  */
/* ------------------------------------------------------------------------ */
double orc_pseudo_angle(double x, double y)
{
    double s = fabs(x) + fabs(y);
    if (s == 0.0) return 0.0;
    double t = x / s;
    return (y >= 0.0) ? 1.0 - t : 3.0 + t;
}

typedef struct {
    double k;
    int i;
} keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *p = (const keyidx *)a, *q = (const keyidx *)b;
    if (p->k < q->k) return -1;
    if (p->k > q->k) return 1;
    return (p->i > q->i) - (p->i < q->i);
}

int orc_default_k(int n)
{
    if (n < 300) return 1;
    if (n < 500) return 3;
    return 5;
}

/* perm[n]: circles in partition order; bounds[k+1]: batch p is perm[bounds[p]..bounds[p+1]).
 * seed, inst: the random partition's Philox key and instance word (other modes ignore them). */
void orc_partition_seeded(int n, const double *xy, int k, int mode, uint64_t seed, int inst, int32_t *perm,
                          int32_t *bounds)
{
    keyidx *a = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    uint32_t pkey[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; i++) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        double key;
        if (mode == 3) {
            uint32_t ctr[4] = {(uint32_t)i, 0u, (uint32_t)inst, 0xC0000000u}, w[4];
            orc_philox4x32_10(ctr, pkey, w);
            key = u53(w[0], w[1]);
        } else if (mode == 1)
            key = sqrt(x * x + y * y);
        else if (mode == 2)
            key = x;
        else
            key = orc_pseudo_angle(x, y);
        a[i].k = key;
        a[i].i = i;
    }
    qsort(a, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int i = 0; i < n; i++) perm[i] = a[i].i;
    free(a);
    int q = n / k, r = n % k;
    bounds[0] = 0;
    for (int p = 0; p < k; p++) bounds[p + 1] = bounds[p] + q + (p < r ? 1 : 0);
}

void orc_partition(int n, const double *xy, int k, int mode, int32_t *perm, int32_t *bounds)
{
    orc_partition_seeded(n, xy, k, mode, 0, 0, perm, bounds);
}

/* ------------------------------------------------------------------------ */
/* Limited-memory inverse Hessian (Eq. 10 / Eq. 11 kept as m secant pairs).  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int m, dim, count, head; /* head: slot of the oldest pair */
    double *S, *Y, *rho;     /* S[m*dim], Y[m*dim], rho[m] */
} lmem;

static void lmem_init(lmem *M, int m, int dim)
{
    M->m = m;
    M->dim = dim;
    M->count = 0;
    M->head = 0;
    M->S = (double *)calloc((size_t)m * (size_t)(dim > 0 ? dim : 1), sizeof(double));
    M->Y = (double *)calloc((size_t)m * (size_t)(dim > 0 ? dim : 1), sizeof(double));
    M->rho = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
}

static void lmem_free(lmem *M)
{
    free(M->S);
    free(M->Y);
    free(M->rho);
}

static double dot(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static void lmem_push(lmem *M, const double *s, const double *y, double sy)
{
    int slot;
    if (M->count < M->m) {
        slot = (M->head + M->count) % M->m;
        M->count++;
    } else {
        slot = M->head;
        M->head = (M->head + 1) % M->m;
    }
    memcpy(M->S + (size_t)slot * M->dim, s, sizeof(double) * (size_t)M->dim);
    memcpy(M->Y + (size_t)slot * M->dim, y, sizeof(double) * (size_t)M->dim);
    M->rho[slot] = 1.0 / sy;
}

/*
 * d = -H g by the two-loop recursion (Nocedal & Wright, Alg. 7.4), H0 = gamma I
 * with gamma = s'y / y'y of the newest pair (gamma = 1 with an empty memory).
 */
static void two_loop(const lmem *M, const double *g, double *d, double *alpha)
{
    int n = M->dim;
    for (int i = 0; i < n; i++) d[i] = g[i];
    for (int c = M->count - 1; c >= 0; c--) {
        int slot = (M->head + c) % M->m;
        const double *s = M->S + (size_t)slot * n, *y = M->Y + (size_t)slot * n;
        double a = M->rho[slot] * dot(s, d, n);
        alpha[c] = a;
        for (int i = 0; i < n; i++) d[i] -= a * y[i];
    }
    double gamma = 1.0;
    if (M->count > 0) {
        int slot = (M->head + M->count - 1) % M->m;
        const double *s = M->S + (size_t)slot * n, *y = M->Y + (size_t)slot * n;
        gamma = dot(s, y, n) / dot(y, y, n);
    }
    for (int i = 0; i < n; i++) d[i] *= gamma;
    for (int c = 0; c < M->count; c++) {
        int slot = (M->head + c) % M->m;
        const double *s = M->S + (size_t)slot * n, *y = M->Y + (size_t)slot * n;
        double b = M->rho[slot] * dot(y, d, n);
        for (int i = 0; i < n; i++) d[i] += (alpha[c] - b) * s[i];
    }
    for (int i = 0; i < n; i++) d[i] = -d[i];
}

/*
 * Test hook: two-loop direction for explicit pairs (S, Y row-major [count][dim],
 * oldest first), and the same direction by the dense update of Eq. 10 / Eq. 11
 * applied pair by pair to H0 = gamma I.
 */
void orc_lbfgs_direction(int dim, int count, const double *S, const double *Y, const double *g, double *d)
{
    lmem M;
    lmem_init(&M, count > 0 ? count : 1, dim);
    for (int c = 0; c < count; c++)
        lmem_push(&M, S + (size_t)c * dim, Y + (size_t)c * dim, dot(S + (size_t)c * dim, Y + (size_t)c * dim, dim));
    double *alpha = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    two_loop(&M, g, d, alpha);
    free(alpha);
    lmem_free(&M);
}

void orc_dense_bfgs_direction(int dim, int count, const double *S, const double *Y, const double *g, double *d)
{
    double *H = (double *)calloc((size_t)dim * dim, sizeof(double));
    double *T = (double *)calloc((size_t)dim * dim, sizeof(double));
    double gamma = 1.0;
    if (count > 0) {
        const double *s = S + (size_t)(count - 1) * dim, *y = Y + (size_t)(count - 1) * dim;
        gamma = dot(s, y, dim) / dot(y, y, dim);
    }
    for (int i = 0; i < dim; i++) H[(size_t)i * dim + i] = gamma;
    for (int c = 0; c < count; c++) {
        const double *u = S + (size_t)c * dim, *v = Y + (size_t)c * dim;
        double beta = dot(v, u, dim); /* Eq. 10 */
        /* Eq. 11: H <- (I - u v'/beta) H (I - v u'/beta) + u u'/beta */
        for (int i = 0; i < dim; i++) { /* T = (I - u v'/beta) H */
            for (int j = 0; j < dim; j++) {
                double acc = 0.0;
                for (int q = 0; q < dim; q++) {
                    double a = ((i == q) ? 1.0 : 0.0) - u[i] * v[q] / beta;
                    acc += a * H[(size_t)q * dim + j];
                }
                T[(size_t)i * dim + j] = acc;
            }
        }
        for (int i = 0; i < dim; i++) { /* H = T (I - v u'/beta) + u u'/beta */
            for (int j = 0; j < dim; j++) {
                double acc = 0.0;
                for (int q = 0; q < dim; q++) {
                    double b = ((q == j) ? 1.0 : 0.0) - v[q] * u[j] / beta;
                    acc += T[(size_t)i * dim + q] * b;
                }
                H[(size_t)i * dim + j] = acc + u[i] * u[j] / beta;
            }
        }
    }
    for (int i = 0; i < dim; i++) {
        double acc = 0.0;
        for (int j = 0; j < dim; j++) acc += H[(size_t)i * dim + j] * g[j];
        d[i] = -acc;
    }
    free(H);
    free(T);
}

/* ------------------------------------------------------------------------ */
/* GBO descent (Algorithm "GBO", Sec. 4.1) with ANM (Algorithm "ANM").        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double l_cut;        /* neighbor cutoff (paper: 4; default here 2.5) */
    double rebuild_disp; /* Verlet half-skin: rebuild when 2 D + step_max > 2 rebuild_disp */
    double step_max;     /* cap on any circle's move in one batch step */
    double e_tol;        /* stop: E <= e_tol */
    double gsum_tol;     /* stop: sum_p |g_p|_2 <= gsum_tol (Algorithm GBO) */
    double c1;           /* Armijo constant */
    double curv_eps;     /* push a pair only if s'y > curv_eps |s| |y| */
    int m;               /* memory pairs */
    int max_iter;        /* sweeps */
    int k;               /* batches (0: by n) */
    int partition;       /* 0 sector, 1 annulus, 2 fence, 3 random */
    int max_trials;      /* backtracking trials per search */
    int anm;             /* 1: ANM deferral rebuilds on */
    int prec32_pred;     /* neighbor predicate in binary32 */
    uint64_t part_seed;  /* random partition (3): Philox key */
    int part_inst;       /* random partition: the instance word of the counter */
    int dense;           /* 1: per-batch BFGS with an explicit inverse Hessian (Eq. 10, Eq. 11) */
} orc_opts;

typedef struct {
    int iters, status, builds, changes, disp_builds, trials, resets, stalls;
    double E, gsum;
} orc_result;

enum { ORC_CONVERGED = 0, ORC_STATIONARY = 1, ORC_STALLED = 2, ORC_MAXITER = 3, ORC_ERROR = 4 };

void orc_default_opts(orc_opts *o)
{
    o->l_cut = 2.5;
    o->rebuild_disp = 0.25;
    o->step_max = 0.1;
    o->e_tol = 1e-20;
    o->gsum_tol = 1e-12;
    o->c1 = 1e-4;
    o->curv_eps = 1e-10;
    o->m = 10;
    o->max_iter = 2000;
    o->k = 0;
    o->partition = 0;
    o->max_trials = 30;
    o->anm = 1;
    o->prec32_pred = 0;
    o->part_seed = 0;
    o->part_inst = 0;
    o->dense = 0;
}

/* The explicit inverse-Hessian approximation of one batch (Eq. 8, Eq. 10, Eq. 11).  It starts as
 * I (the first step is a gradient step); before the first update it is rescaled to
 * (s'y / y'y) I from that first pair, the usual initial scaling of BFGS; each accepted pair with
 * enough curvature then applies Eq. 11, expanded as the symmetric rank-two change
 *   H+ = H - rho (Hy) s' - rho s (Hy)' + (rho^2 y'Hy + rho) s s',  rho = 1 / (y's).
 * A reset returns it to I. */
typedef struct {
    int dim, fresh;
    double *H, *Hy;
} dmem;

static void dmem_reset(dmem *M)
{
    memset(M->H, 0, sizeof(double) * (size_t)M->dim * (size_t)M->dim);
    for (int i = 0; i < M->dim; i++) M->H[(size_t)i * M->dim + i] = 1.0;
    M->fresh = 1;
}

static void dmem_init(dmem *M, int dim)
{
    M->dim = dim;
    M->H = (double *)malloc(sizeof(double) * (size_t)(dim > 0 ? dim : 1) * (size_t)(dim > 0 ? dim : 1));
    M->Hy = (double *)malloc(sizeof(double) * (size_t)(dim > 0 ? dim : 1));
    dmem_reset(M);
}

static void dmem_free(dmem *M)
{
    free(M->H);
    free(M->Hy);
}

static void dmem_update(dmem *M, const double *s, const double *y, double sy, double yy);

/* One update of Eq. 11 on a caller's H (n x n, row major, already scaled): the same code the
 * dense descent runs, for the tests. */
void orc_bfgs_update(int n, double *H, const double *s, const double *y)
{
    double sy = 0.0, yy = 0.0;
    for (int i = 0; i < n; i++) {
        sy += s[i] * y[i];
        yy += y[i] * y[i];
    }
    dmem M;
    M.dim = n;
    M.fresh = 0;
    M.H = H;
    M.Hy = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    dmem_update(&M, s, y, sy, yy);
    free(M.Hy);
}

/* d = -H g */
static void dmem_direction(const dmem *M, const double *g, double *d)
{
    for (int r = 0; r < M->dim; r++) {
        double v = 0.0;
        const double *h = M->H + (size_t)r * M->dim;
        for (int c = 0; c < M->dim; c++) v += h[c] * g[c];
        d[r] = -v;
    }
}

static void dmem_update(dmem *M, const double *s, const double *y, double sy, double yy)
{
    const int n = M->dim;
    if (M->fresh) {
        const double gam = sy / yy;
        memset(M->H, 0, sizeof(double) * (size_t)n * (size_t)n);
        for (int i = 0; i < n; i++) M->H[(size_t)i * n + i] = gam;
        M->fresh = 0;
    }
    double yHy = 0.0;
    for (int r = 0; r < n; r++) {
        double v = 0.0;
        const double *h = M->H + (size_t)r * n;
        for (int c = 0; c < n; c++) v += h[c] * y[c];
        M->Hy[r] = v;
        yHy += y[r] * v;
    }
    const double rho = 1.0 / sy, cs = rho * rho * yHy + rho;
    for (int r = 0; r < n; r++) {
        double *h = M->H + (size_t)r * n;
        for (int c = 0; c < n; c++) h[c] += -rho * (M->Hy[r] * s[c] + s[r] * M->Hy[c]) + cs * s[r] * s[c];
    }
}

typedef struct {
    int32_t *row_ptr, *col;
    int64_t cap, nnz;
} csr;

static int csr_build(csr *c, int n, const double *xy, double R, const orc_opts *o)
{
    for (;;) {
        int64_t r = orc_neighbors_cells(n, xy, R, o->l_cut, o->prec32_pred, c->row_ptr, c->col, c->cap);
        if (r >= 0) {
            c->nnz = r;
            return 0;
        }
        c->cap = -r + 16;
        c->col = (int32_t *)realloc(c->col, sizeof(int32_t) * (size_t)c->cap);
        if (!c->col) return -1;
    }
}

static int csr_equal(const csr *a, const csr *b, int n)
{
    if (a->nnz != b->nnz) return 0;
    if (memcmp(a->row_ptr, b->row_ptr, sizeof(int32_t) * (size_t)(n + 1))) return 0;
    return memcmp(a->col, b->col, sizeof(int32_t) * (size_t)a->nnz) == 0;
}

/*
 * One neighbor (re)construction, ANM bookkeeping included (Algorithm ANM):
 * build Gamma' at the current x; Gamma' == Gamma doubles len, otherwise
 * Gamma <- Gamma' and len <- 1; cnt <- 0.  The layout of the build is kept
 * so the displacement since it can be measured.
 */
static void anm_rebuild(csr *G, csr *Gt, int n, const double *xy, double R, const orc_opts *o,
                        int *cnt, int *len, double *xb, double *D, orc_result *res)
{
    csr_build(Gt, n, xy, R, o);
    res->builds++;
    if (csr_equal(G, Gt, n)) {
        if (*len < (1 << 30)) *len *= 2;
    } else {
        csr t = *G;
        *G = *Gt;
        *Gt = t;
        *len = 1;
        res->changes++;
    }
    *cnt = 0;
    memcpy(xb, xy, sizeof(double) * 2 * (size_t)n);
    *D = 0.0;
}

/*
 * GBO on one instance, in place on xy[2n].  trace (optional, length
 * max_iter+1) receives E after every sweep (trace[0]: the starting E).
 */
int orc_gbo(int n, double *xy, double R, const orc_opts *o, orc_result *res, double *trace)
{
    memset(res, 0, sizeof(*res));
    if (n <= 0) {
        res->status = ORC_CONVERGED;
        return 0;
    }
    int k = o->k > 0 ? o->k : orc_default_k(n);
    if (k > n) k = n;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *bounds = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *batch_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_partition_seeded(n, xy, k, o->partition, o->part_seed, o->part_inst, perm, bounds);
    for (int p = 0; p < k; p++)
        for (int a = bounds[p]; a < bounds[p + 1]; a++) batch_of[perm[a]] = p;

    csr G = {0}, Gt = {0};
    G.cap = Gt.cap = (int64_t)n * 8 + 64;
    G.row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    Gt.row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    G.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)G.cap);
    Gt.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)Gt.cap);
    csr_build(&G, n, xy, R, o);
    res->builds = 1;

    double *xb = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    memcpy(xb, xy, sizeof(double) * 2 * (size_t)n);
    double D = 0.0;
    int cnt = 0, len = 1;

    int maxnb = bounds[1] - bounds[0];
    lmem *mem = (lmem *)malloc(sizeof(lmem) * (size_t)k);
    for (int p = 0; p < k; p++) lmem_init(&mem[p], o->m, 2 * (bounds[p + 1] - bounds[p]));
    dmem *dm = NULL;
    if (o->dense) {
        dm = (dmem *)malloc(sizeof(dmem) * (size_t)k);
        for (int p = 0; p < k; p++) dmem_init(&dm[p], 2 * (bounds[p + 1] - bounds[p]));
    }
    size_t vb = sizeof(double) * 2 * (size_t)maxnb;
    double *g = (double *)malloc(vb), *gn = (double *)malloc(vb), *d = (double *)malloc(vb);
    double *xo = (double *)malloc(vb), *s = (double *)malloc(vb), *y = (double *)malloc(vb);
    double *alpha = (double *)malloc(sizeof(double) * (size_t)(o->m > 0 ? o->m : 1));

    double E = orc_energy_csr(n, xy, R, G.row_ptr, G.col);
    if (trace) trace[0] = E;
    res->status = ORC_MAXITER;
    if (E <= o->e_tol) res->status = ORC_CONVERGED;
    int t = 0;
    while (res->status != ORC_CONVERGED && t < o->max_iter) {
        t++;
        double gsum = 0.0;
        int moved = 0;
        for (int p = 0; p < k; p++) {
            /* Verlet guarantee: a pair missing from Gamma is at least l_cut apart at
             * the build, so it cannot overlap while twice the largest displacement
             * (plus this step's cap) stays within l_cut - 2 = 2 rebuild_disp. */
            if (2.0 * D + o->step_max > 2.0 * o->rebuild_disp) {
                anm_rebuild(&G, &Gt, n, xy, R, o, &cnt, &len, xb, &D, res);
                res->disp_builds++;
            }
            const int32_t *mb = perm + bounds[p];
            int nb = bounds[p + 1] - bounds[p], dim = 2 * nb;
            lmem *M = &mem[p];
            double E0 = orc_batch_energy(xy, R, G.row_ptr, G.col, mb, nb, batch_of, p);
            batch_grad(xy, R, G.row_ptr, G.col, mb, nb, g);
            double gnorm = sqrt(dot(g, g, dim));
            gsum += gnorm;
            if (gnorm == 0.0) continue;
            for (int a = 0; a < nb; a++) {
                xo[2 * a] = xy[2 * mb[a]];
                xo[2 * a + 1] = xy[2 * mb[a] + 1];
            }
            int accepted = 0;
            dmem *DM = dm ? &dm[p] : NULL;
            for (int attempt = 0; attempt < 2 && !accepted; attempt++) {
                if (attempt == 1) {
                    if (DM ? DM->fresh : M->count == 0) break;
                    if (DM) dmem_reset(DM);
                    M->count = 0;
                    M->head = 0;
                    res->resets++;
                }
                if (DM)
                    dmem_direction(DM, g, d);
                else
                    two_loop(M, g, d, alpha);
                double gd = dot(g, d, dim);
                if (!(gd < 0.0)) {
                    if (DM ? !DM->fresh : M->count > 0) {
                        if (DM) dmem_reset(DM);
                        M->count = 0;
                        M->head = 0;
                        res->resets++;
                    }
                    for (int i = 0; i < dim; i++) d[i] = -g[i];
                    gd = -gnorm * gnorm;
                }
                double dmax = 0.0;
                for (int a = 0; a < nb; a++) {
                    double v = sqrt(d[2 * a] * d[2 * a] + d[2 * a + 1] * d[2 * a + 1]);
                    if (v > dmax) dmax = v;
                }
                double al = (dmax > o->step_max) ? o->step_max / dmax : 1.0;
                for (int tr = 0; tr < o->max_trials; tr++) {
                    for (int a = 0; a < nb; a++) {
                        xy[2 * mb[a]] = xo[2 * a] + al * d[2 * a];
                        xy[2 * mb[a] + 1] = xo[2 * a + 1] + al * d[2 * a + 1];
                    }
                    double Et = orc_batch_energy(xy, R, G.row_ptr, G.col, mb, nb, batch_of, p);
                    res->trials++;
                    if (Et <= E0 + o->c1 * al * gd) {
                        accepted = 1;
                        break;
                    }
                    al *= 0.5;
                }
                if (!accepted) {
                    for (int a = 0; a < nb; a++) {
                        xy[2 * mb[a]] = xo[2 * a];
                        xy[2 * mb[a] + 1] = xo[2 * a + 1];
                    }
                }
            }
            if (!accepted) {
                res->stalls++;
                continue;
            }
            moved = 1;
            batch_grad(xy, R, G.row_ptr, G.col, mb, nb, gn);
            double dmv = 0.0;
            for (int a = 0; a < nb; a++) {
                int i = mb[a];
                s[2 * a] = xy[2 * i] - xo[2 * a];
                s[2 * a + 1] = xy[2 * i + 1] - xo[2 * a + 1];
                double ex = xy[2 * i] - xb[2 * i], ey = xy[2 * i + 1] - xb[2 * i + 1];
                double v = sqrt(ex * ex + ey * ey);
                if (v > dmv) dmv = v;
            }
            if (dmv > D) D = dmv;
            for (int i = 0; i < dim; i++) y[i] = gn[i] - g[i];
            double sy = dot(s, y, dim);
            double ns = sqrt(dot(s, s, dim)), ny = sqrt(dot(y, y, dim));
            if (DM) {
                if (sy > o->curv_eps * ns * ny) dmem_update(DM, s, y, sy, ny * ny);
            } else if (M->m > 0 && sy > o->curv_eps * ns * ny) {
                lmem_push(M, s, y, sy);
            }
        }
        /* ANM, called once per sweep (Algorithm GBO). */
        if (o->anm) {
            cnt++;
            if (cnt >= len) anm_rebuild(&G, &Gt, n, xy, R, o, &cnt, &len, xb, &D, res);
        }
        E = orc_energy_csr(n, xy, R, G.row_ptr, G.col);
        if (trace) trace[t] = E;
        res->gsum = gsum;
        if (E <= o->e_tol)
            res->status = ORC_CONVERGED;
        else if (gsum <= o->gsum_tol) {
            res->status = ORC_STATIONARY;
            break;
        } else if (!moved) {
            res->status = ORC_STALLED;
            break;
        }
    }
    res->iters = t;
    res->E = E;

    free(perm);
    free(bounds);
    free(batch_of);
    free(G.row_ptr);
    free(G.col);
    free(Gt.row_ptr);
    free(Gt.col);
    free(xb);
    for (int p = 0; p < k; p++) lmem_free(&mem[p]);
    free(mem);
    if (dm) {
        for (int p = 0; p < k; p++) dmem_free(&dm[p]);
        free(dm);
    }
    free(g);
    free(gn);
    free(d);
    free(xo);
    free(s);
    free(y);
    free(alpha);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Container adjustment (Sec. 4.2, Algorithm adjust_container, Eq. 12).      */
/* ------------------------------------------------------------------------ */
/*
 * U(z, lambda) = E(x, R) + lambda R^2 over the lists and its gradient over z = (x, R):
 * g[0 .. 2n) = dE/dx (grad_row), g[2n] = dU/dR = -2 sum_i d_i0 + 2 lambda R, since
 * d(d_i0^2)/dR = -2 d_i0 for d_i0 = max(0, |c_i| + 1 - R).
 */
static double u_energy_grad(int n, const double *xy, double R, double lambda, const csr *G, double *g)
{
    ksum sd = {0.0, 0.0};
    for (int i = 0; i < n; i++) {
        grad_row(i, xy, R, G->row_ptr, G->col, &g[2 * i], &g[2 * i + 1], NULL);
        ks_add(&sd, bound_depth(xy[2 * i], xy[2 * i + 1], R, NULL));
    }
    g[2 * n] = -2.0 * ks_get(&sd) + 2.0 * lambda * R;
    return orc_energy_csr(n, xy, R, G->row_ptr, G->col) + lambda * R * R;
}

/* U and its gradient on the brute-force lists (for the tests): g[2n + 1]. */
double orc_u_energy_grad(int n, const double *xy, double R, double lambda, double *g)
{
    csr G = {0};
    G.cap = (int64_t)n * (n > 0 ? n : 1);
    G.row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    G.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G.cap > 0 ? G.cap : 1));
    G.nnz = orc_neighbors_brute(n, xy, 2.0, 0, G.row_ptr, G.col, G.cap);
    double U = u_energy_grad(n, xy, R, lambda, &G, g);
    free(G.row_ptr);
    free(G.col);
    return U;
}

/*
 * adjust_container: z = (x, R); for t = 1 .. rounds minimise U(z, lambda) by a
 * limited-memory BFGS over all of z, then halve lambda (lambda starts at lambda0).  Each
 * round starts a fresh memory (U changes with lambda) and runs the descent of GBO with
 * one batch: Armijo search from alpha0 = min(1, step_max / max(max_i |d_i|, |d_R|)), the
 * Verlet rule and ANM on the lists, a pair kept when s'y > curv_eps |s| |y|; a round ends
 * when |g| <= gsum_tol (stationary), when no step is accepted (stalled) or after max_iter
 * iterations.  In place on xy[2n] and *R; res sums the rounds' iterations, builds and
 * trials; status and E (of the final layout and radius) are those after the last round.
 */
int orc_adjust_container(int n, double *xy, double *Rp, const orc_opts *o, double lambda0, int rounds,
                         orc_result *res)
{
    memset(res, 0, sizeof(*res));
    double R = *Rp;
    if (n <= 0) {
        res->status = ORC_CONVERGED;
        return 0;
    }
    const int dim = 2 * n + 1;
    csr G = {0}, Gt = {0};
    G.cap = Gt.cap = (int64_t)n * 8 + 64;
    G.row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    Gt.row_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    G.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)G.cap);
    Gt.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)Gt.cap);
    csr_build(&G, n, xy, R, o);
    res->builds = 1;
    double *xb = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    memcpy(xb, xy, sizeof(double) * 2 * (size_t)n);
    double D = 0.0;
    int cnt = 0, len = 1;
    size_t vb = sizeof(double) * (size_t)dim;
    double *g = (double *)malloc(vb), *gn = (double *)malloc(vb), *d = (double *)malloc(vb);
    double *zo = (double *)malloc(vb), *s = (double *)malloc(vb), *y = (double *)malloc(vb);
    double *alpha = (double *)malloc(sizeof(double) * (size_t)(o->m > 0 ? o->m : 1));
    lmem M;
    lmem_init(&M, o->m, dim);
    double lambda = lambda0;
    int status = ORC_MAXITER;
    for (int round = 0; round < rounds; round++) {
        M.count = 0;
        M.head = 0;
        status = ORC_MAXITER;
        for (int t = 0; t < o->max_iter; t++) {
            if (2.0 * D + o->step_max > 2.0 * o->rebuild_disp) {
                anm_rebuild(&G, &Gt, n, xy, R, o, &cnt, &len, xb, &D, res);
                res->disp_builds++;
            }
            res->iters++;
            double U0 = u_energy_grad(n, xy, R, lambda, &G, g);
            double gnorm = sqrt(dot(g, g, dim));
            if (!(gnorm > o->gsum_tol)) {
                status = ORC_STATIONARY;
                break;
            }
            memcpy(zo, xy, sizeof(double) * 2 * (size_t)n);
            zo[2 * n] = R;
            int accepted = 0;
            for (int attempt = 0; attempt < 2 && !accepted; attempt++) {
                if (attempt == 1) {
                    if (M.count == 0) break;
                    M.count = 0;
                    M.head = 0;
                    res->resets++;
                }
                two_loop(&M, g, d, alpha);
                double gd = dot(g, d, dim);
                if (!(gd < 0.0)) {
                    if (M.count > 0) {
                        M.count = 0;
                        M.head = 0;
                        res->resets++;
                    }
                    for (int i = 0; i < dim; i++) d[i] = -g[i];
                    gd = -gnorm * gnorm;
                }
                double dmax = fabs(d[2 * n]);
                for (int a = 0; a < n; a++) {
                    double v = sqrt(d[2 * a] * d[2 * a] + d[2 * a + 1] * d[2 * a + 1]);
                    if (v > dmax) dmax = v;
                }
                double al = (dmax > o->step_max) ? o->step_max / dmax : 1.0;
                for (int tr = 0; tr < o->max_trials; tr++) {
                    for (int i = 0; i < 2 * n; i++) xy[i] = zo[i] + al * d[i];
                    R = zo[2 * n] + al * d[2 * n];
                    double Ut = orc_energy_csr(n, xy, R, G.row_ptr, G.col) + lambda * R * R;
                    res->trials++;
                    if (Ut <= U0 + o->c1 * al * gd) {
                        accepted = 1;
                        break;
                    }
                    al *= 0.5;
                }
                if (!accepted) {
                    memcpy(xy, zo, sizeof(double) * 2 * (size_t)n);
                    R = zo[2 * n];
                }
            }
            if (!accepted) {
                res->stalls++;
                status = ORC_STALLED;
                break;
            }
            u_energy_grad(n, xy, R, lambda, &G, gn);
            double dmv = 0.0;
            for (int i = 0; i < n; i++) {
                double ex = xy[2 * i] - xb[2 * i], ey = xy[2 * i + 1] - xb[2 * i + 1];
                double v = sqrt(ex * ex + ey * ey);
                if (v > dmv) dmv = v;
            }
            if (dmv > D) D = dmv;
            for (int i = 0; i < 2 * n; i++) s[i] = xy[i] - zo[i];
            s[2 * n] = R - zo[2 * n];
            for (int i = 0; i < dim; i++) y[i] = gn[i] - g[i];
            double sy = dot(s, y, dim);
            double ns = sqrt(dot(s, s, dim)), ny = sqrt(dot(y, y, dim));
            if (M.m > 0 && sy > o->curv_eps * ns * ny) lmem_push(&M, s, y, sy);
            if (o->anm) {
                cnt++;
                if (cnt >= len) anm_rebuild(&G, &Gt, n, xy, R, o, &cnt, &len, xb, &D, res);
            }
        }
        lambda *= 0.5;
    }
    res->status = status;
    res->E = orc_energy_csr(n, xy, R, G.row_ptr, G.col);
    *Rp = R;
    free(G.row_ptr);
    free(G.col);
    free(Gt.row_ptr);
    free(Gt.col);
    free(xb);
    lmem_free(&M);
    free(g);
    free(gn);
    free(d);
    free(zo);
    free(s);
    free(y);
    free(alpha);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Feasibility (Eq. 1, Eq. 2): largest pair depth over all pairs and largest */
/* boundary depth, brute force.  Returns the larger of the two.              */
/* ------------------------------------------------------------------------ */
double orc_max_overlap(int n, const double *xy, double R, double *max_pair, double *max_bound)
{
    double mp = 0.0, mb = 0.0;
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            double s = dx * dx;
            double t = dy * dy;
            s = s + t;
            double d = 2.0 - sqrt(s);
            if (d > mp) mp = d;
        }
        double b = bound_depth(xy[2 * i], xy[2 * i + 1], R, NULL);
        if (b > mb) mb = b;
    }
    if (max_pair) *max_pair = mp;
    if (max_bound) *max_bound = mb;
    return mp > mb ? mp : mb;
}

/* ------------------------------------------------------------------------ */
/* Whole path for many independent instances: init (Sec. 5.1), GBO, and the */
/* feasibility check, instances spread over nthreads POSIX threads.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int num;
    const int32_t *n;
    const double *R;
    const int64_t *offset; /* circle offset of each instance */
    uint64_t seed;
    int inst_base;
    int init_mode;
    const orc_opts *o;
    double feas_tol;
    double *xy;        /* [2 * sum n] final positions */
    int32_t *iters, *status;
    double *E, *max_overlap;
    uint8_t *feasible;
    int next;
    pthread_mutex_t lock;
} solve_job;

static void *solve_worker(void *arg)
{
    solve_job *J = (solve_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int q = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (q >= J->num) break;
        int n = J->n[q];
        double *xy = J->xy + 2 * J->offset[q];
        orc_init_positions(n, J->R[q], J->seed, J->inst_base + q, J->init_mode, xy);
        orc_result r;
        orc_gbo(n, xy, J->R[q], J->o, &r, NULL);
        double mo = orc_max_overlap(n, xy, J->R[q], NULL, NULL);
        J->iters[q] = r.iters;
        J->status[q] = r.status;
        J->E[q] = r.E;
        J->max_overlap[q] = mo;
        J->feasible[q] = (uint8_t)(mo <= J->feas_tol);
    }
    return NULL;
}

/* Returns wall seconds spent (steady clock). */
double orc_solve_batch(int num, const int32_t *n, const double *R, uint64_t seed, int inst_base,
                       int init_mode, const orc_opts *o, double feas_tol, int nthreads, double *xy,
                       int32_t *iters, int32_t *status, double *E, double *max_overlap, uint8_t *feasible)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(num + 1));
    off[0] = 0;
    for (int q = 0; q < num; q++) off[q + 1] = off[q] + n[q];
    solve_job J = {num, n, R, off, seed, inst_base, init_mode, o, feas_tol, xy,
                   iters, status, E, max_overlap, feasible, 0, PTHREAD_MUTEX_INITIALIZER};
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, solve_worker, &J);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    free(th);
    free(off);
    return (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
}

/* ------------------------------------------------------------------------ */
/* SED (Sec. 5.2, Algorithm SED): solution-space exploring and descent at a */
/* fixed container radius.  From the GBO minimum of a random layout, each    */
/* iteration perturbs the operated solution x into m = max(1, J(E(x)))       */
/* candidates, descends each by GBO, and replaces x by the select operator   */
/* of Eq. 18; the best solution x* is kept, and the search stops once        */
/* E(x*) <= e_feas (the paper: 1e-25) or after s_iter iterations.            */
/* Random numbers: Philox4x32-10 with key = seed; candidate j of iteration   */
/* it draws counter (i, it, inst, 2^31 + j) for circle i, the select draw    */
/* counter (0, it, inst, 2^30) (the initial layout uses c3 = 0).             */
/* ------------------------------------------------------------------------ */

/* J(E) = ceil(-log10 E) (Sec. 5.2); +2^30 for E <= 0. */
int orc_sed_J(double E)
{
    if (!(E > 0.0)) return 1 << 30;
    return (int)ceil(-log10(E));
}

/* The perturbation of Sec. 5.2: x'_i = x_i + r, y'_i = y_i + r with r ~ U(-amp, amp), amp = 0.8.
 * shared = 0: r drawn independently for x and for y; shared = 1: one r for both, as printed. */
void orc_sed_perturb(int n, const double *xy, uint64_t seed, int inst, int it, int j, int shared, double amp,
                     double *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; i++) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)inst, 0x80000000u | (uint32_t)j}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double rx = amp * (2.0 * u53(w[0], w[1]) - 1.0);
        double ry = shared ? rx : amp * (2.0 * u53(w[2], w[3]) - 1.0);
        out[2 * i] = xy[2 * i] + rx;
        out[2 * i + 1] = xy[2 * i + 1] + ry;
    }
}

/* select (Eq. 18).  The candidate of least energy when that energy is below E(x) (the first of
 * equal ones).  Otherwise a draw with probability softmax(J(y)): with w_j = exp(J_j - max J),
 * the first j whose running sum w_0 + ... + w_j exceeds u (w_0 + ... + w_{m-1}), u uniform in
 * [0, 1) from the select counter. */
int orc_sed_select(int m, const double *E, double Ex, uint64_t seed, int inst, int it)
{
    if (m <= 1) return 0;
    int best = 0;
    for (int j = 1; j < m; j++)
        if (E[j] < E[best]) best = j;
    if (E[best] < Ex) return best;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {0u, (uint32_t)it, (uint32_t)inst, 0x40000000u}, w[4];
    orc_philox4x32_10(ctr, key, w);
    double u = u53(w[0], w[1]);
    int Jmax = orc_sed_J(E[0]);
    for (int j = 1; j < m; j++) {
        int J = orc_sed_J(E[j]);
        if (J > Jmax) Jmax = J;
    }
    double tot = 0.0;
    for (int j = 0; j < m; j++) tot += exp((double)(orc_sed_J(E[j]) - Jmax));
    double target = u * tot, run = 0.0;
    for (int j = 0; j < m; j++) {
        run += exp((double)(orc_sed_J(E[j]) - Jmax));
        if (target < run) return j;
    }
    return m - 1;
}

typedef struct {
    int iters;     /* SED iterations performed */
    int status;    /* 0: E(x*) <= e_feas; 3: s_iter iterations without reaching it */
    int descents;  /* GBO calls, the initial one included */
    double E0;     /* energy after the initial descent */
    double E;      /* E(x*) */
} orc_sed_result;

/* SED on one instance.  xy_best receives x*.  Traces (length s_iter, may be NULL): per iteration
 * the candidate count m, the selected candidate, E(x) after the selection and E(x*). */
int orc_sed(int n, double R, uint64_t seed, int inst, int init_mode, const orc_opts *o, int s_iter, int max_cand,
            double e_feas, int shared, double amp, double *xy_best, orc_sed_result *res, int32_t *m_trace,
            int32_t *sel_trace, double *Ex_trace, double *Eb_trace)
{
    memset(res, 0, sizeof(*res));
    size_t vb = sizeof(double) * 2 * (size_t)(n > 0 ? n : 1);
    double *x = (double *)malloc(vb);
    double *cand = (double *)malloc(vb * (size_t)(max_cand > 0 ? max_cand : 1));
    double *Ec = (double *)malloc(sizeof(double) * (size_t)(max_cand > 0 ? max_cand : 1));
    orc_result r;
    orc_init_positions(n, R, seed, inst, init_mode, x);
    orc_gbo(n, x, R, o, &r, NULL);
    res->descents = 1;
    double Ex = r.E, Eb = r.E;
    res->E0 = r.E;
    memcpy(xy_best, x, sizeof(double) * 2 * (size_t)n);
    int it = 0;
    for (; it < s_iter; it++) {
        if (Eb <= e_feas) break;
        int m = orc_sed_J(Ex);
        if (m < 1) m = 1;
        if (m > max_cand) m = max_cand;
        for (int j = 0; j < m; j++) {
            double *c = cand + (size_t)j * 2 * (size_t)n;
            orc_sed_perturb(n, x, seed, inst, it, j, shared, amp, c);
            orc_gbo(n, c, R, o, &r, NULL);
            Ec[j] = r.E;
            res->descents++;
        }
        int sel = orc_sed_select(m, Ec, Ex, seed, inst, it);
        memcpy(x, cand + (size_t)sel * 2 * (size_t)n, sizeof(double) * 2 * (size_t)n);
        Ex = Ec[sel];
        if (Ex < Eb) {
            Eb = Ex;
            memcpy(xy_best, x, sizeof(double) * 2 * (size_t)n);
        }
        if (m_trace) m_trace[it] = m;
        if (sel_trace) sel_trace[it] = sel;
        if (Ex_trace) Ex_trace[it] = Ex;
        if (Eb_trace) Eb_trace[it] = Eb;
    }
    res->iters = it;
    res->E = Eb;
    res->status = Eb <= e_feas ? ORC_CONVERGED : ORC_MAXITER;
    free(x);
    free(cand);
    free(Ec);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The framework of Sec. 5.1 (Algorithm 5) with an iteration count in place  */
/* of the cut-off time: x* = GBO(random_solution(n, R_b)), (x*, R*) =        */
/* adjust(x*, R_b); then `outer` times: R = min(R_b, R*), x = SED(n, R),     */
/* (x, R) = adjust(x, R), and x*, R* = x, R when R < R*.  Random keys: the   */
/* first layout draws under `seed`, SED call t under seed + 1 + t.  The GBO  */
/* and SED stop at e_feas.  R_trace (outer + 1, may be NULL): R* after      */
/* the first adjustment and after every iteration.                           */
/* ------------------------------------------------------------------------ */
int orc_frame(int n, double Rb, uint64_t seed, int inst, int init_mode, const orc_opts *o, int outer, int s_iter,
              int max_cand, double e_feas, double amp, double lambda0, int rounds, double *xy_best, double *R_best,
              double *R_trace)
{
    size_t vb = sizeof(double) * 2 * (size_t)(n > 0 ? n : 1);
    double *x = (double *)malloc(vb);
    orc_result r;
    orc_opts os = *o;
    os.e_tol = e_feas;
    orc_init_positions(n, Rb, seed, inst, init_mode, x);
    orc_gbo(n, x, Rb, &os, &r, NULL);
    double Rs = Rb;
    orc_adjust_container(n, x, &Rs, o, lambda0, rounds, &r);
    memcpy(xy_best, x, sizeof(double) * 2 * (size_t)n);
    if (R_trace) R_trace[0] = Rs;
    for (int t = 0; t < outer; t++) {
        const double R = Rb < Rs ? Rb : Rs;
        orc_sed_result sr;
        orc_sed(n, R, seed + 1 + (uint64_t)t, inst, init_mode, &os, s_iter, max_cand, e_feas, 0, amp, x, &sr, NULL,
                NULL, NULL, NULL);
        double Rn = R;
        orc_adjust_container(n, x, &Rn, o, lambda0, rounds, &r);
        if (Rn < Rs) {
            Rs = Rn;
            memcpy(xy_best, x, sizeof(double) * 2 * (size_t)n);
        }
        if (R_trace) R_trace[t + 1] = Rs;
    }
    *R_best = Rs;
    free(x);
    return 0;
}
