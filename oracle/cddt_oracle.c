/*
 * cddt_oracle.c -- the CPU oracle for CDDT ray casting and the beam sensor
 * model (Walsh & Karaman, "CDDT: Fast Approximate 2D Ray Casting for
 * Accelerated Localization", arXiv 1705.01167).
 *
 * TEST INFRASTRUCTURE.  This file is not part of the product.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * It is written to be plain, slow and checkable against the paper by eye:
 *   O1  brute force: one query scans every edge cell of the map (no bins kept)
 *   O2  plain CDDT: per-bin growable arrays filled in the order of the
 *       construction algorithm (Section IV-A), each bin sorted afterwards,
 *       queried with a textbook successor / predecessor binary search
 *       (Section IV-B, Section IV-C)
 *   O3  exact voxel-traversal caster (Amanatides & Woo, 1987), a
 *       Bresenham caster and a ray marcher over a distance transform
 *       (Section II), for approximation reports and the baselines
 *   O4  tiny-map lookup table, every discrete state cast by O1 (Section II)
 *   O5  FP64 beam sensor model, its log-weight and its analytic gradient
 *   prune (Section IV-C) and incremental update (Section IV-D)
 *
 * Parity unpinned: the choices the paper leaves open and no outside fact
 * fixes -- lambda_short = 0.01 and the other beam-model constants, the
 * truncated-normal option of p_hit, range 0 for an off-map query (S6), and
 * the 16-bit scheme's Q and X_s (S7).  Every function below is pinned by the
 * CPU tests to the paper's worked example, closed forms, library routines,
 * brute force or invariants; these choices are only held equal on both
 * sides.
 *
 * Floating-point contract: the CDDT geometry is float32 with an explicit
 * operation order and no contraction (build with -ffp-contract=off); the
 * beam model is float64.  The readings taken where the paper is silent:
 *
 *  S0  cell (i, j) is grid[j*W + i], centred on the integer point (i, j) and
 *      covering [i-1/2, i+1/2) x [j-1/2, j+1/2); theta runs from +x toward +y.
 *  S1  N directions over the full circle, theta_k = 2 pi k / N; a query's k is
 *      round-half-up(theta * N/(2 pi)) wrapped into [0, N); only slices
 *      s < N/2 are stored and k >= N/2 searches slice k - N/2 backwards
 *      (the theta / theta + pi symmetry, Section IV-C).
 *  S2  slice trig (cos, sin)(2 pi s / N) evaluated in double, rounded to
 *      float, snapped to (1, 0) at s = 0 and (0, 1) at s = N/4.
 *  S3  projection: xr = x*c + y*s; yr = y*c - x*s (float32, products first,
 *      then the sum).  The translation that makes bin indices non-negative is
 *      an integer T_s added after rounding: bin = floor(yr + 1/2) + T_s, with
 *      T_s = ceil(-min corner yr) + 1 and nbins_s = ceil(max corner yr + T_s)
 *      + 2 over the map's four corners.
 *  S4  a cell's rotated square spans yr +- h, h = (|c| + |s|)/2; bin b - T_s
 *      covers [b - T_s - 1/2, b - T_s + 1/2); a cell enters every bin whose
 *      open interval meets (yr - h, yr + h); a query uses bin
 *      floor(yr + 1/2) + T_s.
 *  S5  forward = first zero point > x'; backward = last zero point < x';
 *      duplicate zero points are kept (bins are multisets).
 *  S6  a query whose nearest cell is off the map or occupied returns 0; no
 *      zero point in the search direction returns max_range; otherwise
 *      min(range, max_range).  Zero points come from the edge map
 *      (occupied cells with at least one free or off-map 8-neighbour).
 *  S7  16-bit zero points: Q = 2^floor(log2(65535/(diag + 4))), per-slice
 *      integer offset X_s = ceil(-min corner xr) + 1, key = floor((xr + X_s)
 *      * Q + 1/2), value = key / Q - X_s (exact in float32).
 *  S8  pruning keeps zero point z_m of bin (s, b) iff the closed gap
 *      [z_{m-1}, z_m] or [z_m, z_{m+1}] meets the x'-extent of some free
 *      in-map cell whose y'-extent meets bin b, both extents widened by eps.
 *  S9  beam model: p = z_hit p_hit + z_short p_short + z_max p_max + z_rand
 *      p_rand (Probabilistic Robotics, beam model), weight = sum of log p.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ params */

typedef struct {
    int32_t W, H, N, nsl, full, u16;
    float max_range;
    double Q;          /* u16 scale (power of two), 0 when u16 is off */
    float *c, *s;      /* per slice cos / sin (S2)                    */
    int32_t *T;        /* per slice integer bin offset                */
    float *X;          /* per slice x offset for u16 (integer-valued) */
    int32_t *nb;       /* bins per slice                              */
    int64_t *sbase;    /* first global bin of each slice, nsl + 1     */
    int64_t total_bins;
} oc_params;

typedef struct {
    oc_params *p;
    uint8_t *grid, *edge;
    int32_t *len, *cap;
    float **bin;
    int pruned;
} oc_cddt;

void oc_params_free(oc_params *p)
{
    if (!p) return;
    free(p->c); free(p->s); free(p->T); free(p->X); free(p->nb); free(p->sbase);
    free(p);
}

/* Slice tables (S1-S3, S7).  full = 1 stores all N directions (used only by
 * the symmetry check); full = 0 stores the N/2 slices of Section IV-C. */
oc_params *oc_params_new(int32_t W, int32_t H, int32_t N, float max_range, int32_t u16,
                         int32_t full)
{
    if (W < 1 || H < 1 || N < 2 || (N % 2) != 0) return NULL;
    oc_params *p = (oc_params *)calloc(1, sizeof(oc_params));
    p->W = W; p->H = H; p->N = N; p->full = full; p->u16 = u16;
    p->max_range = max_range;
    p->nsl = full ? N : N / 2;
    p->c = (float *)malloc(sizeof(float) * p->nsl);
    p->s = (float *)malloc(sizeof(float) * p->nsl);
    p->T = (int32_t *)malloc(sizeof(int32_t) * p->nsl);
    p->X = (float *)malloc(sizeof(float) * p->nsl);
    p->nb = (int32_t *)malloc(sizeof(int32_t) * p->nsl);
    p->sbase = (int64_t *)malloc(sizeof(int64_t) * (p->nsl + 1));
    if (u16) {
        double diag = sqrt((double)W * W + (double)H * H);
        double q = 65535.0 / (diag + 4.0);
        int e;
        if (q < 1.0) { oc_params_free(p); return NULL; }
        frexp(q, &e);               /* q = m 2^e, m in [0.5, 1) */
        p->Q = ldexp(1.0, e - 1);   /* 2^floor(log2 q) */
    }
    double cx[4] = {-0.5, W - 0.5, -0.5, W - 0.5};
    double cy[4] = {-0.5, -0.5, H - 0.5, H - 0.5};
    p->sbase[0] = 0;
    for (int32_t sl = 0; sl < p->nsl; ++sl) {
        double ang = (2.0 * OC_PI * (double)sl) / (double)N;
        float c = (float)cos(ang), s = (float)sin(ang);
        if (sl == 0) { c = 1.0f; s = 0.0f; }
        if (4 * sl == N) { c = 0.0f; s = 1.0f; }
        if (full && 2 * sl == N) { c = -1.0f; s = 0.0f; }
        if (full && 4 * sl == 3 * N) { c = 0.0f; s = -1.0f; }
        p->c[sl] = c; p->s[sl] = s;
        double ymin = 1e300, ymax = -1e300, xmin = 1e300;
        for (int q = 0; q < 4; ++q) {
            double yr = cy[q] * (double)c - cx[q] * (double)s;
            double xr = cx[q] * (double)c + cy[q] * (double)s;
            if (yr < ymin) ymin = yr;
            if (yr > ymax) ymax = yr;
            if (xr < xmin) xmin = xr;
        }
        double T = ceil(-ymin) + 1.0;
        p->T[sl] = (int32_t)T;
        p->nb[sl] = (int32_t)(ceil(ymax + T) + 2.0);
        p->X[sl] = (float)(ceil(-xmin) + 1.0);
        p->sbase[sl + 1] = p->sbase[sl] + p->nb[sl];
    }
    p->total_bins = p->sbase[p->nsl];
    return p;
}

void oc_params_export(const oc_params *p, float *c, float *s, int32_t *T, float *X,
                      int32_t *nb, int64_t *sbase, double *Q)
{
    memcpy(c, p->c, sizeof(float) * p->nsl);
    memcpy(s, p->s, sizeof(float) * p->nsl);
    memcpy(T, p->T, sizeof(int32_t) * p->nsl);
    memcpy(X, p->X, sizeof(float) * p->nsl);
    memcpy(nb, p->nb, sizeof(int32_t) * p->nsl);
    memcpy(sbase, p->sbase, sizeof(int64_t) * (p->nsl + 1));
    *Q = p->Q;
}

int32_t oc_params_nsl(const oc_params *p) { return p->nsl; }
int64_t oc_params_total_bins(const oc_params *p) { return p->total_bins; }

/* ------------------------------------------------------------ geometry */

/* Edge map (Section IV-A erosion, Section IV-C): an occupied cell is an edge
 * cell unless all eight neighbours are occupied; off-map counts as free. */
static int is_edge(const uint8_t *g, int W, int H, int i, int j)
{
    if (!g[(int64_t)j * W + i]) return 0;
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            if (!di && !dj) continue;
            int a = i + di, b = j + dj;
            if (a < 0 || a >= W || b < 0 || b >= H) return 1;
            if (!g[(int64_t)b * W + a]) return 1;
        }
    return 0;
}

void oc_edge_map(const uint8_t *grid, int32_t W, int32_t H, uint8_t *edge)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) edge[(int64_t)j * W + i] = (uint8_t)is_edge(grid, W, H, i, j);
}

/* Projection P_DDT (S3): the rotation by -theta_s; the translation is the
 * integer bin offset T_s applied where a bin index is formed. */
static void project(const oc_params *p, int sl, float x, float y, float *xr, float *yr)
{
    float c = p->c[sl], s = p->s[sl];
    float a = x * c;
    float b = y * s;
    *xr = a + b;
    float ya = y * c;
    float yb2 = x * s;
    *yr = ya - yb2;
}

/* Bin of a query at rotated ordinate yr (S4). */
static int query_bin(const oc_params *p, int sl, float yr)
{
    return (int)floorf(yr + 0.5f) + p->T[sl];
}

static float half_extent(const oc_params *p, int sl)
{
    float t = fabsf(p->c[sl]) + fabsf(p->s[sl]);
    return 0.5f * t;
}

/* Bins whose open interval meets the open y'-extent of a cell (S4). */
static int cell_bins(const oc_params *p, int sl, float yr, int *bmin, int *bmax)
{
    float h = half_extent(p, sl);
    float lo = yr - h;
    lo = lo - 0.5f;
    float hi = yr + h;
    hi = hi + 0.5f;
    int a = (int)floorf(lo) + 1 + p->T[sl];
    int b = (int)ceilf(hi) - 1 + p->T[sl];
    if (a < 0) a = 0;
    if (b > p->nb[sl] - 1) b = p->nb[sl] - 1;
    *bmin = a; *bmax = b;
    return a <= b;
}

/* The stored value of a zero point: xr itself, or its 16-bit rounding (S7). */
static float store_value(const oc_params *p, int sl, float xr)
{
    if (!p->u16) return xr;
    float u = xr + p->X[sl];
    float v = u * (float)p->Q;
    float w = v + 0.5f;
    float key = floorf(w);
    if (key < 0.0f) key = 0.0f;
    if (key > 65535.0f) key = 65535.0f;
    return key * (float)(1.0 / p->Q) - p->X[sl];
}

/* Query direction (S1): slice index, search direction; returns 0 when theta
 * is not finite. */
static int query_slice(const oc_params *p, float theta, int *sl, int *backward)
{
    float inv_step = (float)((double)p->N / (2.0 * OC_PI));
    float t = theta * inv_step;
    float tk = floorf(t + 0.5f);
    if (!isfinite(tk)) return 0;
    float km = fmodf(tk, (float)p->N);
    int k = (int)km;
    if (k < 0) k += p->N;
    if (p->full) { *sl = k; *backward = 0; }
    else if (k >= p->N / 2) { *sl = k - p->N / 2; *backward = 1; }
    else { *sl = k; *backward = 0; }
    return 1;
}

int32_t oc_query_k(const oc_params *p, float theta)
{
    float inv_step = (float)((double)p->N / (2.0 * OC_PI));
    float t = theta * inv_step;
    float tk = floorf(t + 0.5f);
    if (!isfinite(tk)) return -1;
    float km = fmodf(tk, (float)p->N);
    int k = (int)km;
    if (k < 0) k += p->N;
    return k;
}

/* Occupancy pre-check (S6): 1 when the query may be cast. */
static int free_cell(const oc_params *p, const uint8_t *grid, float x, float y)
{
    float fx = floorf(x + 0.5f), fy = floorf(y + 0.5f);
    if (!(fx >= 0.0f && fx < (float)p->W && fy >= 0.0f && fy < (float)p->H)) return 0;
    return grid[(int64_t)fy * p->W + (int64_t)fx] == 0;
}

/* ------------------------------------------------------------ O2 build */

static void bin_append(oc_cddt *d, int64_t g, float v)
{
    if (d->len[g] == d->cap[g]) {
        int32_t nc = d->cap[g] ? 2 * d->cap[g] : 4;
        d->bin[g] = (float *)realloc(d->bin[g], sizeof(float) * nc);
        d->cap[g] = nc;
    }
    d->bin[g][d->len[g]++] = v;
}

static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Direct construction (Section IV-A): edge map; for every slice, every edge
 * cell is projected and appended to each bin it overlaps; each bin is then
 * sorted (the sorted-vector successor structure of Section IV-B). */
oc_cddt *oc_build(const uint8_t *grid, int32_t W, int32_t H, int32_t N, float max_range,
                  int32_t u16, int32_t full)
{
    oc_params *p = oc_params_new(W, H, N, max_range, u16, full);
    if (!p) return NULL;
    oc_cddt *d = (oc_cddt *)calloc(1, sizeof(oc_cddt));
    d->p = p;
    int64_t n = (int64_t)W * H;
    d->grid = (uint8_t *)malloc(n);
    for (int64_t q = 0; q < n; ++q) d->grid[q] = grid[q] ? 1 : 0;
    d->edge = (uint8_t *)malloc(n);
    oc_edge_map(d->grid, W, H, d->edge);
    d->len = (int32_t *)calloc(p->total_bins, sizeof(int32_t));
    d->cap = (int32_t *)calloc(p->total_bins, sizeof(int32_t));
    d->bin = (float **)calloc(p->total_bins, sizeof(float *));
    for (int sl = 0; sl < p->nsl; ++sl) {
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                if (!d->edge[(int64_t)j * W + i]) continue;
                float xr, yr;
                int b0, b1;
                project(p, sl, (float)i, (float)j, &xr, &yr);
                if (!cell_bins(p, sl, yr, &b0, &b1)) continue;
                float v = store_value(p, sl, xr);
                for (int b = b0; b <= b1; ++b) bin_append(d, p->sbase[sl] + b, v);
            }
        for (int b = 0; b < p->nb[sl]; ++b) {
            int64_t g = p->sbase[sl] + b;
            if (d->len[g] > 1) qsort(d->bin[g], d->len[g], sizeof(float), cmp_float);
        }
    }
    return d;
}

void oc_free(oc_cddt *d)
{
    if (!d) return;
    for (int64_t g = 0; g < d->p->total_bins; ++g) free(d->bin[g]);
    free(d->bin); free(d->len); free(d->cap); free(d->grid); free(d->edge);
    oc_params_free(d->p);
    free(d);
}

const oc_params *oc_get_params(const oc_cddt *d) { return d->p; }

int64_t oc_total_zp(const oc_cddt *d)
{
    int64_t t = 0;
    for (int64_t g = 0; g < d->p->total_bins; ++g) t += d->len[g];
    return t;
}

/* Flatten to CSR: bin_start[total_bins + 1], zp[total]. */
void oc_export(const oc_cddt *d, int64_t *bin_start, float *zp)
{
    int64_t o = 0;
    for (int64_t g = 0; g < d->p->total_bins; ++g) {
        bin_start[g] = o;
        if (d->len[g]) memcpy(zp + o, d->bin[g], sizeof(float) * d->len[g]);
        o += d->len[g];
    }
    bin_start[d->p->total_bins] = o;
}

void oc_export_grid(const oc_cddt *d, uint8_t *grid, uint8_t *edge)
{
    int64_t n = (int64_t)d->p->W * d->p->H;
    memcpy(grid, d->grid, n);
    memcpy(edge, d->edge, n);
}

/* ------------------------------------------------------------ O2 query */

/* Textbook successor search: index of the first element > x, or n. */
static int32_t upper_bound_f(const float *a, int32_t n, float x)
{
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Textbook search: index of the first element >= x, or n. */
static int32_t lower_bound_f(const float *a, int32_t n, float x)
{
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* One ray cast through the plain CDDT (Section IV-B query, Section IV-C
 * backward search).  *kb receives the size of the bin searched (-1 when no
 * bin is searched), *zi the index of the zero point used (-1 for none). */
static float o2_cast(const oc_cddt *d, float x, float y, float theta, int32_t *kb, int32_t *zi,
                     int32_t *sl_out, int32_t *bin_out)
{
    const oc_params *p = d->p;
    *kb = -1; *zi = -1; *sl_out = -1; *bin_out = -1;
    if (!free_cell(p, d->grid, x, y)) return 0.0f;
    int sl, bwd;
    if (!query_slice(p, theta, &sl, &bwd)) return 0.0f;
    float xq, yq;
    project(p, sl, x, y, &xq, &yq);
    int b = query_bin(p, sl, yq);
    *sl_out = sl; *bin_out = b;
    if (b < 0 || b >= p->nb[sl]) return p->max_range;
    int64_t g = p->sbase[sl] + b;
    const float *a = d->bin[g];
    int32_t n = d->len[g];
    *kb = n;
    float r;
    if (!bwd) {
        int32_t i = upper_bound_f(a, n, xq);
        if (i == n) return p->max_range;
        *zi = i;
        r = a[i] - xq;
    } else {
        int32_t i = lower_bound_f(a, n, xq) - 1;
        if (i < 0) return p->max_range;
        *zi = i;
        r = xq - a[i];
    }
    return fminf(r, p->max_range);
}

void oc_calc_range(const oc_cddt *d, const float *pose, int64_t n, float *out, int32_t nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int32_t kb, zi, sl, b;
        out[q] = o2_cast(d, pose[3 * q], pose[3 * q + 1], pose[3 * q + 2], &kb, &zi, &sl, &b);
    }
}

/* Per-query instrumentation: bin size searched, zero-point index, slice, bin. */
void oc_calc_range_info(const oc_cddt *d, const float *pose, int64_t n, float *out,
                        int32_t *kb, int32_t *zi, int32_t *sl, int32_t *bin)
{
    for (int64_t q = 0; q < n; ++q)
        out[q] = o2_cast(d, pose[3 * q], pose[3 * q + 1], pose[3 * q + 2], kb + q, zi + q,
                         sl + q, bin + q);
}

/* ------------------------------------------------------------ O1 brute force */

/* The same query answered from the definition: every edge cell of the map is
 * projected into the query's slice; those overlapping the query's bin are the
 * bin's zero points; take the nearest one strictly beyond x' in the search
 * direction.  No bin is stored or sorted. */
static float o1_cast(const oc_params *p, const uint8_t *grid, const uint8_t *edge, float x,
                     float y, float theta)
{
    if (!free_cell(p, grid, x, y)) return 0.0f;
    int sl, bwd;
    if (!query_slice(p, theta, &sl, &bwd)) return 0.0f;
    float xq, yq;
    project(p, sl, x, y, &xq, &yq);
    int b = query_bin(p, sl, yq);
    if (b < 0 || b >= p->nb[sl]) return p->max_range;
    int found = 0;
    float best = 0.0f;
    for (int j = 0; j < p->H; ++j)
        for (int i = 0; i < p->W; ++i) {
            if (!edge[(int64_t)j * p->W + i]) continue;
            float xr, yr;
            int b0, b1;
            project(p, sl, (float)i, (float)j, &xr, &yr);
            if (!cell_bins(p, sl, yr, &b0, &b1) || b < b0 || b > b1) continue;
            float v = store_value(p, sl, xr);
            if (!bwd) {
                if (v > xq && (!found || v < best)) { best = v; found = 1; }
            } else {
                if (v < xq && (!found || v > best)) { best = v; found = 1; }
            }
        }
    if (!found) return p->max_range;
    float r = bwd ? xq - best : best - xq;
    return fminf(r, p->max_range);
}

void oc_calc_range_brute(const oc_params *p, const uint8_t *grid, const float *pose, int64_t n,
                         float *out, int32_t nthreads)
{
    int64_t cells = (int64_t)p->W * p->H;
    uint8_t *g = (uint8_t *)malloc(cells), *e = (uint8_t *)malloc(cells);
    for (int64_t q = 0; q < cells; ++q) g[q] = grid[q] ? 1 : 0;
    oc_edge_map(g, p->W, p->H, e);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q)
        out[q] = o1_cast(p, g, e, pose[3 * q], pose[3 * q + 1], pose[3 * q + 2]);
    free(g); free(e);
}

/* The zero-point multiset of one bin from the definition (sorted): used to
 * check single bins of maps too large to build here in full. */
int32_t oc_bin_brute(const oc_params *p, const uint8_t *grid, int32_t sl, int32_t b, float *out,
                     int32_t cap)
{
    int32_t n = 0;
    for (int j = 0; j < p->H; ++j)
        for (int i = 0; i < p->W; ++i) {
            if (!is_edge(grid, p->W, p->H, i, j)) continue;
            float xr, yr;
            int b0, b1;
            project(p, sl, (float)i, (float)j, &xr, &yr);
            if (!cell_bins(p, sl, yr, &b0, &b1) || b < b0 || b > b1) continue;
            if (n < cap) out[n] = store_value(p, sl, xr);
            ++n;
        }
    if (n <= cap && n > 1) qsort(out, n, sizeof(float), cmp_float);
    return n;
}

/* ------------------------------------------------------------ O4 tiny LUT */

/* The three-dimensional lookup table of Section II: every discrete state
 * (cell centre, theta_k) cast by O1.  out[(k*H + j)*W + i]. */
void oc_lut(const oc_params *p, const uint8_t *grid, float *out)
{
    for (int k = 0; k < p->N; ++k) {
        float th = (float)((2.0 * OC_PI * (double)k) / (double)p->N);
        for (int j = 0; j < p->H; ++j)
            for (int i = 0; i < p->W; ++i) {
                float pose[3] = {(float)i, (float)j, th};
                oc_calc_range_brute(p, grid, pose, 1, out + ((int64_t)k * p->H + j) * p->W + i, 1);
            }
    }
}

/* ------------------------------------------------------------ O3 casters */

/* Exact ray cast on the continuous ray (no theta rounding) by voxel traversal
 * (Amanatides & Woo).  Returns, for the first occupied cell met, the distance
 * along the ray to its centre's projection (mode 0) or to the ray's entry
 * point into the cell (mode 1).  Start cell occupied or off map: 0.  No hit
 * within max_range: max_range. */
void oc_cast_exact(const uint8_t *grid, int32_t W, int32_t H, const double *pose, int64_t n,
                   double max_range, int32_t mode, double *out)
{
    for (int64_t q = 0; q < n; ++q) {
        double x = pose[3 * q], y = pose[3 * q + 1], th = pose[3 * q + 2];
        long i = (long)floor(x + 0.5), j = (long)floor(y + 0.5);
        if (i < 0 || i >= W || j < 0 || j >= H || grid[(int64_t)j * W + i]) { out[q] = 0.0; continue; }
        double dx = cos(th), dy = sin(th);
        int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1;
        double tdx = dx != 0 ? fabs(1.0 / dx) : INFINITY;
        double tdy = dy != 0 ? fabs(1.0 / dy) : INFINITY;
        double bx = sx > 0 ? (i + 0.5) : (i - 0.5);
        double by = sy > 0 ? (j + 0.5) : (j - 0.5);
        double tmx = dx != 0 ? (bx - x) / dx : INFINITY;
        double tmy = dy != 0 ? (by - y) / dy : INFINITY;
        double res = max_range;
        for (;;) {
            double tenter;
            if (tmx < tmy) { i += sx; tenter = tmx; tmx += tdx; }
            else { j += sy; tenter = tmy; tmy += tdy; }
            if (tenter > max_range) break;
            if (i < 0 || i >= W || j < 0 || j >= H) break;
            if (grid[(int64_t)j * W + i]) {
                res = mode ? tenter : (i - x) * dx + (j - y) * dy;
                if (res > max_range) res = max_range;
                break;
            }
        }
        out[q] = res;
    }
}

/* Bresenham's line (Section II): integer steps from the query cell toward the
 * point max_range away; Euclidean distance to the first occupied pixel. */
/* Direction of a continuous heading for the Bresenham and ray marching
 * casters (reading D1), float32, one rounding per operation:
 *   1. |theta| > 2^16: theta = fmodf(theta, fl(2 pi))   (exact remainder)
 *   2. j = rint(theta * fl(2/pi)); r = theta - j pi/2, with pi/2 split into
 *      three floats P1 + P2 + P3 and one fused multiply-add per part
 *      (Cody & Waite's additive reduction)
 *   3. sin r = r + r^3 (-1/3! + r^2 (1/5! + r^2 (-1/7! + r^2 / 9!))),
 *      cos r = 1 + r^2 (-1/2! + r^2 (1/4! + r^2 (-1/6! + r^2 (1/8! - r^2 / 10!)))),
 *      each bracket one fused multiply-add, coefficients fl(1/n!)
 *   4. quadrant j mod 4: (sin, cos) = (s, c), (c, -s), (-s, -c), (-c, s). */
void oc_dir_sincos(float th, float *sin_out, float *cos_out)
{
    const float P1 = 0x1.921fb6p+0f, P2 = -0x1.777a5cp-25f, P3 = -0x1.ee59dap-50f;
    if (fabsf(th) > 65536.0f) th = fmodf(th, 0x1.921fb6p+2f);
    float j = rintf(th * 0x1.45f306p-1f);
    float r = fmaf(-j, P1, th);
    r = fmaf(-j, P2, r);
    r = fmaf(-j, P3, r);
    float r2 = r * r;
    float sp = fmaf(fmaf(fmaf(r2, 1.0f / 362880.0f, -1.0f / 5040.0f), r2, 1.0f / 120.0f), r2, -1.0f / 6.0f);
    float sr = fmaf(r2 * r, sp, r);
    float cp = fmaf(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    cp = fmaf(r2, cp, -1.0f / 720.0f);
    cp = fmaf(r2, cp, 1.0f / 24.0f);
    cp = fmaf(r2, cp, -0.5f);
    float cr = fmaf(r2, cp, 1.0f);
    switch ((int)j & 3) {
    case 0: *sin_out = sr; *cos_out = cr; break;
    case 1: *sin_out = cr; *cos_out = -sr; break;
    case 2: *sin_out = -sr; *cos_out = -cr; break;
    default: *sin_out = -cr; *cos_out = sr; break;
    }
}

/* Bresenham's line caster (Section II), float32 query and arithmetic: the
 * digital line from the query's cell floor(p + 1/2) to the cell
 * floor(p + max_range (c, s) + 1/2) (one fused multiply-add per coordinate;
 * c, s by oc_dir_sincos) by integer error stepping; the range is the
 * distance from the query point to the first occupied cell's centre, at
 * most max_range.  0 for a non-finite coordinate or a start cell that is
 * occupied or off the map (as a CDDT query, S6); max_range when the walk
 * leaves the map or reaches its end. */
void oc_cast_bresenham(const uint8_t *grid, int32_t W, int32_t H, const float *pose, int64_t n, float max_range,
                       float *out)
{
    for (int64_t q = 0; q < n; ++q) {
        float x = pose[3 * q], y = pose[3 * q + 1], th = pose[3 * q + 2];
        if (!isfinite(th) || !isfinite(x) || !isfinite(y)) { out[q] = 0.0f; continue; }
        float fx0 = floorf(x + 0.5f), fy0 = floorf(y + 0.5f);
        if (!(fx0 >= 0.0f && fx0 < (float)W && fy0 >= 0.0f && fy0 < (float)H) ||
            grid[(int64_t)fy0 * W + (int64_t)fx0]) { out[q] = 0.0f; continue; }
        float s, c;
        oc_dir_sincos(th, &s, &c);
        long long x0 = (long long)fx0, y0 = (long long)fy0;
        long long x1 = (long long)floorf(fmaf(max_range, c, x) + 0.5f);
        long long y1 = (long long)floorf(fmaf(max_range, s, y) + 0.5f);
        long long ddx = llabs(x1 - x0), ddy = -llabs(y1 - y0);
        int sx = x0 < x1 ? 1 : -1, sy = y0 < y1 ? 1 : -1;
        long long err = ddx + ddy, cx = x0, cy = y0;
        float res = max_range;
        while (!(cx == x1 && cy == y1)) {
            long long e2 = 2 * err;
            if (e2 >= ddy) { err += ddy; cx += sx; }
            if (e2 <= ddx) { err += ddx; cy += sy; }
            if (cx < 0 || cx >= W || cy < 0 || cy >= H) break;
            if (grid[(int64_t)cy * W + cx]) {
                float dx = (float)cx - x, dy = (float)cy - y;
                res = sqrtf(dx * dx + dy * dy);
                if (res > max_range) res = max_range;
                break;
            }
        }
        out[q] = res;
    }
}

/* Ray marching (Section II, reading RM1) over a distance transform E, float
 * [H][W], E[j*W + i] the distance from cell (i, j)'s centre to the nearest
 * occupied cell's centre (0 on occupied cells).  float32 throughout, the
 * sample point by explicit fmaf: from t = 0, read the cell under
 * (x + t c, y + t s); stop off the map (max_range) or on an occupied cell
 * (t); else advance t by the distance read, stopping at max_range.  c, s
 * come from oc_dir_sincos.  0 for a non-finite
 * coordinate or a start off the map.  steps[q] = distance reads of ray q. */
void oc_raymarch(const float *E, int32_t W, int32_t H, const float *pose, int64_t n, float max_range,
                 float *out, int32_t *steps)
{
    for (int64_t q = 0; q < n; ++q) {
        float x = pose[3 * q], y = pose[3 * q + 1], th = pose[3 * q + 2];
        float res = 0.0f;
        int32_t reads = 0;
        if (isfinite(x) && isfinite(y) && isfinite(th)) {
            float fx = floorf(x + 0.5f), fy = floorf(y + 0.5f);
            if (fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H) {
                float s, c;
                oc_dir_sincos(th, &s, &c);
                float t = 0.0f;
                res = max_range;
                for (;;) {
                    fx = floorf(fmaf(t, c, x) + 0.5f);
                    fy = floorf(fmaf(t, s, y) + 0.5f);
                    if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) break;
                    float d = E[(int64_t)fy * W + (int64_t)fx];
                    ++reads;
                    if (d == 0.0f) { res = t; break; }
                    t = t + d;
                    if (!(t < max_range)) break;
                }
            }
        }
        out[q] = res;
        steps[q] = reads;
    }
}

/* ------------------------------------------------------------ O5 beam model */

typedef struct {
    float z_hit, z_short, z_max, z_rand, sigma_hit, lambda_short, max_range;
    int32_t hit_truncnorm;
} oc_beam_model;

static double std_normal_cdf(double u) { return 0.5 * (1.0 + erf(u / sqrt(2.0))); }
static double std_normal_pdf(double u) { return exp(-0.5 * u * u) / sqrt(2.0 * OC_PI); }

/* Mixture density p(z | z*) of the beam model and dp/dz*.  z is the measured
 * range clamped to [0, max_range], zs the expected range. */
static void beam_p(const oc_beam_model *m, double z, double zs, double *p_out, double *dp_out)
{
    double zmax = m->max_range, sig = m->sigma_hit, lam = m->lambda_short;
    if (z < 0.0) z = 0.0;
    if (z > zmax) z = zmax;
    double d = z - zs;
    double p_hit = exp(-(d * d) / (2.0 * sig * sig)) / (sig * sqrt(2.0 * OC_PI));
    double dp_hit = p_hit * d / (sig * sig);
    if (m->hit_truncnorm) {
        double a = (zmax - zs) / sig, b = -zs / sig;
        double D = std_normal_cdf(a) - std_normal_cdf(b);
        double dD = (std_normal_pdf(b) - std_normal_pdf(a)) / sig;
        p_hit = p_hit / D;
        dp_hit = p_hit * (d / (sig * sig) - dD / D);
    }
    double p_short = 0.0, dp_short = 0.0;
    if (zs > 0.0 && z <= zs) {
        double den = 1.0 - exp(-lam * zs);
        p_short = lam * exp(-lam * z) / den;
        if (z < zs) dp_short = -lam * lam * exp(-lam * z) * exp(-lam * zs) / (den * den);
    }
    double p_max = z >= zmax ? 1.0 : 0.0;
    double p_rand = z < zmax ? 1.0 / zmax : 0.0;
    *p_out = m->z_hit * p_hit + m->z_short * p_short + m->z_max * p_max + m->z_rand * p_rand;
    *dp_out = m->z_hit * dp_hit + m->z_short * dp_short;
}

void oc_beam_eval(const oc_beam_model *m, const double *z, const double *zs, int64_t n,
                  double *p, double *dp)
{
    for (int64_t q = 0; q < n; ++q) beam_p(m, z[q], zs[q], p + q, dp + q);
}

/* Log-weight of every particle: log w_p = sum over beams of log p(z_i | z*_i),
 * z*_i = O2 ray cast from (x, y) at theta_p + phi_i (one float32 add).
 * ranges (P x B) may be NULL. */
void oc_sensor_weights(const oc_cddt *d, const float *part, int64_t P, const float *beam_off,
                       const float *obs, int32_t B, const oc_beam_model *m, double *logw,
                       float *ranges, int32_t nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < P; ++q) {
        float x = part[3 * q], y = part[3 * q + 1], th = part[3 * q + 2];
        double acc = 0.0;
        for (int32_t i = 0; i < B; ++i) {
            int32_t kb, zi, sl, b;
            float a = th + beam_off[i];
            float r = o2_cast(d, x, y, a, &kb, &zi, &sl, &b);
            if (ranges) ranges[q * B + i] = r;
            double pv, dpv;
            beam_p(m, (double)obs[i], (double)r, &pv, &dpv);
            acc += log(pv);
        }
        logw[q] = acc;
    }
}

/* The adjoint: d log w_p / d(x, y) = grad_logw_p * sum_i (dp_i/dz*_i / p_i)
 * dz*_i/d(x, y).  With x' = x c + y s, a forward hit has z* = z - x' and
 * the derivative of z* by (x, y) is -(c, s); a backward hit has z* = x' - z
 * and derivative +(c, s).  The
 * derivative is zero for a clamped range (>= max_range), a miss, or a
 * particle whose cell is occupied or off the map; d/dtheta is zero almost
 * everywhere because theta is rounded to a slice. */
void oc_sensor_grad(const oc_cddt *d, const float *part, int64_t P, const float *beam_off,
                    const float *obs, int32_t B, const oc_beam_model *m, const double *grad_logw,
                    double *grad_xy, double *abs_terms, int32_t nthreads)
{
    const oc_params *p = d->p;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < P; ++q) {
        float x = part[3 * q], y = part[3 * q + 1], th = part[3 * q + 2];
        double gx = 0.0, gy = 0.0, ax = 0.0, ay = 0.0;
        for (int32_t i = 0; i < B; ++i) {
            int32_t kb, zi, sl, b;
            float a = th + beam_off[i];
            float r = o2_cast(d, x, y, a, &kb, &zi, &sl, &b);
            if (zi < 0 || !(r < p->max_range)) continue;
            int s2, bwd;
            query_slice(p, a, &s2, &bwd);
            double dzx = bwd ? (double)p->c[sl] : -(double)p->c[sl];
            double dzy = bwd ? (double)p->s[sl] : -(double)p->s[sl];
            double pv, dpv;
            beam_p(m, (double)obs[i], (double)r, &pv, &dpv);
            double w = dpv / pv;
            gx += w * dzx; gy += w * dzy;
            ax += fabs(w * dzx); ay += fabs(w * dzy);
        }
        grad_xy[2 * q] = grad_logw[q] * gx;
        grad_xy[2 * q + 1] = grad_logw[q] * gy;
        if (abs_terms) {
            abs_terms[2 * q] = fabs(grad_logw[q]) * ax;
            abs_terms[2 * q + 1] = fabs(grad_logw[q]) * ay;
        }
    }
}

/* The same log-weight as a float64 function of a continuous (x, y) for the
 * finite-difference check: every discrete choice (cell, slice, bin, zero
 * point) is taken by the float32 path at ((float)x, (float)y), and the range
 * is then evaluated in float64 as z - (x c + y s) (or its negation), a linear
 * function of (x, y) on each piece.  *state receives a hash of every
 * discrete choice, including the clamp and the short-range indicator, so a
 * sample can be rejected when a choice changes inside the stencil.  grad
 * receives the analytic float64 gradient of the same function. */
double oc_logw_piecewise(const oc_cddt *d, double x, double y, float th, const float *beam_off,
                         const float *obs, int32_t B, const oc_beam_model *m, uint64_t *state,
                         double *grad)
{
    const oc_params *p = d->p;
    float xf = (float)x, yf = (float)y;
    uint64_t h = 1469598103934665603ULL;
#define OC_MIX(v) do { h ^= (uint64_t)(int64_t)(v); h *= 1099511628211ULL; } while (0)
    double acc = 0.0, gx = 0.0, gy = 0.0;
    int ok = free_cell(p, d->grid, xf, yf);
    OC_MIX(ok);
    for (int32_t i = 0; i < B; ++i) {
        float a = th + beam_off[i];
        double zs;
        double dzx = 0.0, dzy = 0.0;
        int32_t kb = -1, zi = -1, sl = -1, b = -1;
        int bwd = 0;
        if (!ok) zs = 0.0;
        else {
            float r = o2_cast(d, xf, yf, a, &kb, &zi, &sl, &b);
            int s2;
            query_slice(p, a, &s2, &bwd);
            if (zi < 0) zs = (double)r;
            else {
                double c = p->c[sl], s = p->s[sl];
                double xp = x * c + y * s;
                double z = (double)d->bin[p->sbase[sl] + b][zi];
                double r64 = bwd ? xp - z : z - xp;
                if (r64 < (double)p->max_range) {
                    zs = r64;
                    dzx = bwd ? c : -c;
                    dzy = bwd ? s : -s;
                } else zs = (double)p->max_range;
                OC_MIX(r64 < (double)p->max_range);
            }
        }
        OC_MIX(sl); OC_MIX(b); OC_MIX(zi); OC_MIX(bwd);
        double zc = obs[i] < 0.0f ? 0.0 : (obs[i] > m->max_range ? m->max_range : obs[i]);
        OC_MIX(zs > 0.0 && zc <= zs);
        OC_MIX(zs > 0.0 && zc < zs);
        double pv, dpv;
        beam_p(m, (double)obs[i], zs, &pv, &dpv);
        acc += log(pv);
        gx += dpv / pv * dzx;
        gy += dpv / pv * dzy;
    }
#undef OC_MIX
    *state = h;
    grad[0] = gx; grad[1] = gy;
    return acc;
}

/* Traversal count of one particle with the theta / theta + pi pairing of
 * Section IV-C: beam i and beam i + D share one search when their slices are
 * the same stored slice in opposite directions. */
int32_t oc_traversals(const oc_params *p, float th, const float *beam_off, int32_t B, int32_t D)
{
    int32_t t = B;
    if (D <= 0) return t;
    for (int32_t i = 0; i + D < B && i < D; ++i) {
        int32_t ki = oc_query_k(p, th + beam_off[i]);
        int32_t kj = oc_query_k(p, th + beam_off[i + D]);
        if (ki >= 0 && kj >= 0 && kj == (ki + p->N / 2) % p->N) --t;
    }
    return t;
}

/* ------------------------------------------------------------ prune (S8) */

static void mark_gaps(const float *a, int32_t M, float lo, float hi, uint8_t *keep)
{
    /* Forward gap of m is [a[m-1], a[m]] (a[-1] = -inf); backward gap of m is
     * [a[m], a[m+1]] (a[M] = +inf).  Either meeting [lo, hi] keeps m.  The
     * forward gaps meeting it are m in [lower_bound(lo), upper_bound(hi)];
     * the backward ones m in [lower_bound(lo) - 1, upper_bound(hi) - 1]. */
    int32_t l = lower_bound_f(a, M, lo);
    int32_t u = upper_bound_f(a, M, hi);
    int32_t m0 = l - 1 < 0 ? 0 : l - 1;
    int32_t m1 = u > M - 1 ? M - 1 : u;
    for (int32_t m = m0; m <= m1; ++m) keep[m] = 1;
}

/* Bins a query from free cell (i, j) of slice sl can use (S8).  In slice 0
 * the rotation is exact (yr = y) and the query bin floor(y + 1/2) + T_0 is
 * computed exactly as the pre-check's row, so row j reaches bin j + T_0 only.
 * Elsewhere the closed y'-extent of the cell, widened by eps, meets bin b's
 * closed interval. */
static void free_cell_bins(const oc_params *p, int sl, int j, float yr, float eps, int *b0,
                           int *b1)
{
    int a, b;
    if (sl == 0 && !p->full) {
        a = b = j + p->T[0];
    } else {
        float h = half_extent(p, sl);
        float lo = (yr - h) - eps, hi = (yr + h) + eps;
        a = (int)ceilf(lo - 0.5f) + p->T[sl];
        b = (int)floorf(hi + 0.5f) + p->T[sl];
    }
    if (a < 0) a = 0;
    if (b > p->nb[sl] - 1) b = p->nb[sl] - 1;
    *b0 = a; *b1 = b;
}

/* Prune (Section IV-C, reading S8): drop every zero point that no query from
 * a free cell can return.  Returns the number of zero points removed, or -1
 * when the handle is already pruned. */
int64_t oc_prune(oc_cddt *d, float eps)
{
    oc_params *p = d->p;
    if (d->pruned) return -1;
    uint8_t **keep = (uint8_t **)calloc(p->total_bins, sizeof(uint8_t *));
    for (int64_t g = 0; g < p->total_bins; ++g)
        keep[g] = (uint8_t *)calloc(d->len[g] ? d->len[g] : 1, 1);
    for (int sl = 0; sl < p->nsl; ++sl) {
        float h = half_extent(p, sl);
        for (int j = 0; j < p->H; ++j)
            for (int i = 0; i < p->W; ++i) {
                if (d->grid[(int64_t)j * p->W + i]) continue;
                float xr, yr;
                int b0, b1;
                project(p, sl, (float)i, (float)j, &xr, &yr);
                free_cell_bins(p, sl, j, yr, eps, &b0, &b1);
                float lo = (xr - h) - eps, hi = (xr + h) + eps;
                for (int b = b0; b <= b1; ++b) {
                    int64_t g = p->sbase[sl] + b;
                    if (d->len[g]) mark_gaps(d->bin[g], d->len[g], lo, hi, keep[g]);
                }
            }
    }
    int64_t removed = 0;
    for (int64_t g = 0; g < p->total_bins; ++g) {
        int32_t o = 0;
        for (int32_t m = 0; m < d->len[g]; ++m)
            if (keep[g][m]) d->bin[g][o++] = d->bin[g][m];
        removed += d->len[g] - o;
        d->len[g] = o;
        free(keep[g]);
    }
    free(keep);
    d->pruned = 1;
    return removed;
}

/* The same rule for one bin, scanning every free cell of the map: keep[m]
 * for the sorted zero points a[0..M) of bin (sl, b). */
void oc_prune_bin(const oc_params *p, const uint8_t *grid, int32_t sl, int32_t b, const float *a,
                  int32_t M, float eps, uint8_t *keep)
{
    memset(keep, 0, M);
    float h = half_extent(p, sl);
    for (int j = 0; j < p->H; ++j)
        for (int i = 0; i < p->W; ++i) {
            if (grid[(int64_t)j * p->W + i]) continue;
            float xr, yr;
            int b0, b1;
            project(p, sl, (float)i, (float)j, &xr, &yr);
            free_cell_bins(p, sl, j, yr, eps, &b0, &b1);
            if (b < b0 || b > b1) continue;
            mark_gaps(a, M, (xr - h) - eps, (xr + h) + eps, keep);
        }
}

/* ------------------------------------------------------------ update (S11) */

static int bin_insert(oc_cddt *d, int64_t g, float v)
{
    bin_append(d, g, v);
    float *a = d->bin[g];
    int32_t k = d->len[g] - 1;
    while (k > 0 && a[k - 1] > v) { a[k] = a[k - 1]; --k; }
    a[k] = v;
    return 0;
}

static int bin_remove(oc_cddt *d, int64_t g, float v)
{
    float *a = d->bin[g];
    for (int32_t k = 0; k < d->len[g]; ++k)
        if (a[k] == v) {
            memmove(a + k, a + k + 1, sizeof(float) * (d->len[g] - k - 1));
            d->len[g]--;
            return 0;
        }
    return 1;
}

/* Incremental update (Section IV-D): cell writes apply in order.  A write
 * that changes a cell re-evaluates the edge status of the cell and its eight
 * neighbours (obstacles revealed or hidden by the erosion); every cell whose
 * edge status flips inserts or removes its zero point in every bin it
 * overlaps, in every slice.  Returns 0, -1 on a pruned handle, or the number
 * of failed removals (an internal inconsistency). */
int64_t oc_update(oc_cddt *d, const int32_t *xy, const uint8_t *occ, int64_t n)
{
    oc_params *p = d->p;
    if (d->pruned) return -1;
    int64_t bad = 0;
    for (int64_t t = 0; t < n; ++t) {
        int x = xy[2 * t], y = xy[2 * t + 1];
        if (x < 0 || x >= p->W || y < 0 || y >= p->H) continue;
        uint8_t nv = occ[t] ? 1 : 0;
        if (d->grid[(int64_t)y * p->W + x] == nv) continue;
        d->grid[(int64_t)y * p->W + x] = nv;
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                int i = x + di, j = y + dj;
                if (i < 0 || i >= p->W || j < 0 || j >= p->H) continue;
                uint8_t e = (uint8_t)is_edge(d->grid, p->W, p->H, i, j);
                if (e == d->edge[(int64_t)j * p->W + i]) continue;
                d->edge[(int64_t)j * p->W + i] = e;
                for (int sl = 0; sl < p->nsl; ++sl) {
                    float xr, yr;
                    int b0, b1;
                    project(p, sl, (float)i, (float)j, &xr, &yr);
                    if (!cell_bins(p, sl, yr, &b0, &b1)) continue;
                    float v = store_value(p, sl, xr);
                    for (int b = b0; b <= b1; ++b) {
                        int64_t g = p->sbase[sl] + b;
                        if (e) bin_insert(d, g, v);
                        else bad += bin_remove(d, g, v);
                    }
                }
            }
    }
    return bad;
}

int32_t oc_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
