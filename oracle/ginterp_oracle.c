/*
 * G-Interp CPU oracle: a plain, slow, single-threaded restatement of the
 * cuSZ-i interpolation predictor-quantizer (arXiv 2312.05492, Sec. IV) and
 * its inverse.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's shared library; the CUDA
 * product path never does, and the two share no code.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (no FMA contraction, IEEE float32/float64, default round-to-nearest-even).
 *
 * Notation (z, y, x), x fastest; i = (z*ny + y)*nx + x.  Axis ids 0=z, 1=y,
 * 2=x.  Level index l = 0, 1, ... for strides s = 1, 2, 4, ... (the paper's
 * level ell = l + 1).  Per-level arrays (e, twoe, inv2e) are indexed by l.
 *
 * Chunk geometry (Sec. IV-A): 8^3 chunks in 3-D, 16^2 in 2-D, 512 points in
 * 1-D.  An ndim-D field is held as dims {nz, ny, nx}; its last ndim axes are
 * chunked with anchor stride A = 8, 16 or 512 and interpolated at strides
 * A/2, ..., 1 (3, 4 or 9 levels); the leading axes hold independent slices
 * (2-D) or rows (1-D): every index along them is an anchor coordinate and
 * nothing is interpolated along them.  level_kind has three entries; levels
 * coarser than stride 4 follow level_kind[2].
 *
 * Readings of the paper taken here:
 *   - neighbour domain is the closed 8^3 chunk [8*floor(n/8), min(.+8, n_d-1)]
 *     along the interpolation axis (Sec. IV-A, Fig. 3); optionally, along x, the
 *     closed 32-point block [32*floor(n/32), min(.+32, n_x-1)] of the GPU
 *     design's 32x8x8 data blocks (Sec. IV-C: four 8^3 chunks share their points
 *     along x).  Anchors stay on the stride-8 grid either way;
 *   - the axis processed later in a level covers the whole finer grid (Fig. 3);
 *   - reconstruction from the integer code: x' = p + (float)(code - R) * 2e;
 *   - the cubic splines divide their integer-weighted sums by the printed
 *     denominators: 16 for not-a-knot (a power of two, so the same as a
 *     multiply by 0.0625) and 40 for the natural cubic (an IEEE division).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* Threads of the OpenMP build (points of one pass in parallel); the plain build
 * always runs on one.  Returns the number of threads that will be used. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* stencil kinds (also the values of the kind map) */
enum { K_ANCHOR = 0, K_COPY = 1, K_LINEAR = 2, K_QUAD_LEFT = 3, K_QUAD_RIGHT = 4,
       K_CUBIC_NAK = 5, K_CUBIC_NATURAL = 6 };

/* ---- Eq. 1: error-bound reduction factor alpha = A(eps) (Sec. IV-B.2) ---- */
double orc_alpha(double eps)
{
    if (eps >= 1e-1) return 2.0;
    if (eps >= 1e-2) return 1.75 + 0.25 * (eps - 1e-2) / (1e-1 - 1e-2);
    if (eps >= 1e-3) return 1.5 + 0.25 * (eps - 1e-3) / (1e-2 - 1e-3);
    if (eps >= 1e-4) return 1.25 + 0.25 * (eps - 1e-4) / (1e-3 - 1e-4);
    if (eps >= 1e-5) return 1.0 + 0.25 * (eps - 1e-5) / (1e-4 - 1e-5);
    return 1.0;
}

/* ---- level-wise error bound e_ell = e / alpha^(ell-1) (Sec. IV-B.1) ----
 * Level l=0 is stride 1 (finest, the full bound); coarser levels get tighter
 * bounds.  alpha powers are formed by repeated multiplication in double. */
void orc_level_bounds(double eb_abs, double alpha, int32_t nlev, float *e, float *twoe, float *inv2e)
{
    double apow = 1.0;
    for (int l = 0; l < nlev; ++l) {
        e[l] = (float)(eb_abs / apow);
        twoe[l] = 2.0f * e[l];
        inv2e[l] = (float)(1.0 / (2.0 * (double)e[l]));
        apow *= alpha;
    }
}

/* ---- chunk geometry (Sec. IV-A) ---- */
static int64_t chunk_edge(int ndim) { return ndim == 1 ? 512 : ndim == 2 ? 16 : 8; }

int32_t orc_levels(int32_t ndim) { return ndim == 1 ? 9 : ndim == 2 ? 4 : 3; }

/* anchor stride per axis: the chunk edge on the last ndim axes, 1 before them */
static void anchor_strides(int ndim, int64_t A[3])
{
    for (int a = 0; a < 3; ++a) A[a] = (a >= 3 - ndim) ? chunk_edge(ndim) : 1;
}

/* ---- value range over finite values (Sec. IV-B.1, data profiling) ----
 * Returns the number of non-finite values; vmin/vmax cover finite values only
 * (both 0 when there is none). */
int64_t orc_value_range(const float *x, int64_t n, float *vmin, float *vmax)
{
    int64_t nonfinite = 0;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        float v = x[i];
        if (!isfinite(v)) { ++nonfinite; continue; }
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    if (lo > hi) { lo = 0.0f; hi = 0.0f; }
    *vmin = lo;
    *vmax = hi;
    return nonfinite;
}

/* absolute bound from a value-range-relative one: eps * (vmax - vmin) */
double orc_rel_to_abs(double eps, float vmin, float vmax)
{
    return eps * ((double)vmax - (double)vmin);
}

/* ---- anchor grid (Sec. IV-A): points whose chunked coordinates are all
 * multiples of the chunk edge ---- */
static int64_t anchors_along(int64_t n, int64_t a) { return (n - 1) / a + 1; }

int64_t orc_anchor_count(int64_t nz, int64_t ny, int64_t nx, int32_t ndim)
{
    int64_t A[3];
    anchor_strides(ndim, A);
    return anchors_along(nz, A[0]) * anchors_along(ny, A[1]) * anchors_along(nx, A[2]);
}

/* ---- 1-D splines (Sec. IV-B.1).  m3, m1, p1, p3 are x_{n-3s}, x_{n-s},
 * x_{n+s}, x_{n+3s}; each expression is evaluated as written, one rounding
 * per operation. ---- */
float orc_spline(int kind, float m3, float m1, float p1, float p3)
{
    switch (kind) {
    case K_COPY:          return m1;
    case K_LINEAR:        return (m1 + p1) * 0.5f;
    case K_QUAD_LEFT:     return ((6.0f * m1 - m3) + 3.0f * p1) * 0.125f;   /* -1/8, 6/8, 3/8 */
    case K_QUAD_RIGHT:    return ((3.0f * m1 + 6.0f * p1) - p3) * 0.125f;   /* 3/8, 6/8, -1/8 */
    case K_CUBIC_NAK:     return (9.0f * (m1 + p1) - (m3 + p3)) * 0.0625f;  /* -1, 9, 9, -1 over 16 */
    case K_CUBIC_NATURAL: return (23.0f * (m1 + p1) - 3.0f * (m3 + p3)) / 40.0f; /* -3, 23, 23, -3 over 40 */
    default:              return NAN;
    }
}

/* ---- pass membership (Sec. IV-A): a non-anchor point belongs to level l,
 * the largest l < L with every chunked coordinate a multiple of s = 2^l, and,
 * within the level, to the pass of the LAST chunked axis in dim order whose
 * coordinate is an odd multiple of s.  Returns the pass id 3*(L-1-l)+k (coarse
 * first), or -1 for an anchor. ---- */
static int pass_of(const int64_t c[3], const int order[3], const int64_t A[3], int L, int *axis, int *level)
{
    int anchor = 1;
    for (int a = 0; a < 3; ++a)
        if (A[a] > 1 && c[a] % A[a] != 0) anchor = 0;
    if (anchor) return -1;
    int l = L - 1;
    for (; l > 0; --l) {
        int64_t s = (int64_t)1 << l;
        int all = 1;
        for (int a = 0; a < 3; ++a)
            if (A[a] > 1 && c[a] % s != 0) all = 0;
        if (all) break;
    }
    int64_t s = (int64_t)1 << l;
    for (int k = 2; k >= 0; --k) {
        int a = order[k];
        if (A[a] > 1 && c[a] % (2 * s) == s) {
            *axis = a;
            *level = l;
            return 3 * (L - 1 - l) + k;
        }
    }
    return -2; /* unreachable for a non-anchor point */
}

/* Stencil kind from the neighbour-count rule (Sec. IV-B.1) within the closed
 * neighbour domain of `dom` points along the interpolation axis (8: the chunk;
 * 32: the x-extended block). */
static int stencil_kind(int64_t n, int64_t s, int64_t nd, int spline, int cubic_kind, int64_t dom)
{
    int64_t lo = dom * (n / dom);
    int64_t hi = lo + dom;
    if (hi > nd - 1) hi = nd - 1;
    int has_m3 = (n - 3 * s >= lo);
    int has_p1 = (n + s <= hi);
    int has_p3 = (n + 3 * s <= hi);
    /* n - s >= lo always holds for a predicted point */
    if (!has_p1) return K_COPY;
    if (!spline) return K_LINEAR;
    if (has_m3 && has_p3) return cubic_kind ? K_CUBIC_NATURAL : K_CUBIC_NAK;
    if (has_m3) return K_QUAD_LEFT;
    if (has_p3) return K_QUAD_RIGHT;
    return K_LINEAR;
}

/* Shared traversal state of compress / decompress / debug prediction. */
typedef struct {
    int64_t dims[3];
    int64_t A[3];     /* anchor stride per axis (1: not chunked, not interpolated) */
    int64_t dom[3];   /* neighbour domain along each axis: the chunk edge, or 32 along x */
    int L;            /* levels: strides 2^(L-1) .. 1 */
    int order[3];
    int level_kind[3];
    int cubic_kind[3];
} sched_t;

static int sched_init(sched_t *S, int64_t nz, int64_t ny, int64_t nx, const int32_t order[3],
                      const int32_t level_kind[3], const int32_t cubic_kind[3], int32_t domain_x, int32_t ndim)
{
    if (ndim < 1 || ndim > 3) return -1;
    if (domain_x == 32 && ndim != 3) return -1;
    S->dims[0] = nz; S->dims[1] = ny; S->dims[2] = nx;
    anchor_strides(ndim, S->A);
    for (int a = 0; a < 3; ++a) S->dom[a] = S->A[a];
    if (domain_x == 32) S->dom[2] = 32;
    S->L = orc_levels(ndim);
    for (int a = 0; a < 3; ++a) {
        S->order[a] = order[a];
        S->level_kind[a] = level_kind[a];
        S->cubic_kind[a] = cubic_kind[a];
    }
    return 0;
}

static int level_kind_of(const sched_t *S, int l) { return S->level_kind[l < 2 ? l : 2]; }

/* Per-point schedule: pass id (255 for anchors) and stencil kind. */
int orc_schedule_maps(int64_t nz, int64_t ny, int64_t nx, const int32_t order[3],
                      const int32_t level_kind[3], const int32_t cubic_kind[3], int32_t domain_x, int32_t ndim,
                      uint8_t *pass_map, uint8_t *kind_map)
{
    sched_t S;
    if (sched_init(&S, nz, ny, nx, order, level_kind, cubic_kind, domain_x, ndim)) return -1;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = (z * ny + y) * nx + x;
                int64_t c[3] = {z, y, x};
                int axis = 0, level = 0;
                int p = pass_of(c, S.order, S.A, S.L, &axis, &level);
                if (p < 0) {
                    pass_map[i] = 255;
                    kind_map[i] = K_ANCHOR;
                    continue;
                }
                pass_map[i] = (uint8_t)p;
                kind_map[i] = (uint8_t)stencil_kind(c[axis], (int64_t)1 << level, S.dims[axis],
                                                    level_kind_of(&S, level), S.cubic_kind[axis], S.dom[axis]);
            }
    return 0;
}

/* A prediction read an undefined value (a broken schedule). */
static void flag_bad(int *bad) { __atomic_store_n(bad, 1, __ATOMIC_RELAXED); }

/* Prediction of point c (level l, axis d) from array v (reconstructed values,
 * or original values in the debug mode).  known (optional) flags which
 * entries of v are already defined; a read of an undefined entry sets *bad. */
static float predict_point(const sched_t *S, const float *v, const uint8_t *known,
                           const int64_t c[3], int d, int l, int *kind_out, int *bad)
{
    int64_t s = (int64_t)1 << l;
    int64_t stride_d = (d == 2) ? 1 : (d == 1) ? S->dims[2] : S->dims[1] * S->dims[2];
    int64_t i = (c[0] * S->dims[1] + c[1]) * S->dims[2] + c[2];
    int kind = stencil_kind(c[d], s, S->dims[d], level_kind_of(S, l), S->cubic_kind[d], S->dom[d]);
    float m3 = 0.0f, m1, p1 = 0.0f, p3 = 0.0f;
    int64_t im1 = i - s * stride_d, ip1 = i + s * stride_d;
    int64_t im3 = i - 3 * s * stride_d, ip3 = i + 3 * s * stride_d;
    m1 = v[im1];
    if (known && !known[im1]) flag_bad(bad);
    if (kind != K_COPY) {
        p1 = v[ip1];
        if (known && !known[ip1]) flag_bad(bad);
    }
    if (kind == K_QUAD_LEFT || kind == K_CUBIC_NAK || kind == K_CUBIC_NATURAL) {
        m3 = v[im3];
        if (known && !known[im3]) flag_bad(bad);
    }
    if (kind == K_QUAD_RIGHT || kind == K_CUBIC_NAK || kind == K_CUBIC_NATURAL) {
        p3 = v[ip3];
        if (known && !known[ip3]) flag_bad(bad);
    }
    *kind_out = kind;
    return orc_spline(kind, m3, m1, p1, p3);
}

/* Visit the points of pass (l, k) in ascending linear index: coordinate along
 * d = order[k] is an odd multiple of s, chunked axes before d in the order are on
 * the s-grid, those after d on the 2s-grid; unchunked axes take every index. */
typedef void (*visit_fn)(void *ctx, const int64_t c[3], int d, int l);

static void for_each_in_pass(const sched_t *S, int l, int k, visit_fn fn, void *ctx)
{
    int64_t s = (int64_t)1 << l;
    int d = S->order[k];
    int64_t start[3], step[3];
    for (int j = 0; j < 3; ++j) {
        int a = S->order[j];
        if (S->A[a] == 1) { start[a] = 0; step[a] = 1; }
        else if (j == k) { start[a] = s; step[a] = 2 * s; }
        else if (j < k) { start[a] = 0; step[a] = s; }
        else { start[a] = 0; step[a] = 2 * s; }
    }
    /* The points of one pass read only points of earlier passes and write only
     * themselves, so the OpenMP build may split the outermost loop among threads
     * (results identical to the single-threaded build). */
    const int64_t n0 = S->dims[0] > start[0] ? (S->dims[0] - start[0] + step[0] - 1) / step[0] : 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i0 = 0; i0 < n0; ++i0) {
        int64_t c[3];
        c[0] = start[0] + i0 * step[0];
        for (c[1] = start[1]; c[1] < S->dims[1]; c[1] += step[1])
            for (c[2] = start[2]; c[2] < S->dims[2]; c[2] += step[2])
                fn(ctx, c, d, l);
    }
}

static void for_each_pass(const sched_t *S, visit_fn fn, void *ctx)
{
    for (int l = S->L - 1; l >= 0; --l)   /* strides 2^(L-1), ..., 2, 1 */
        for (int k = 0; k < 3; ++k)       /* chunked axes in dim order */
            if (S->A[S->order[k]] > 1) for_each_in_pass(S, l, k, fn, ctx);
}

static int64_t lin(const sched_t *S, const int64_t c[3])
{
    return (c[0] * S->dims[1] + c[1]) * S->dims[2] + c[2];
}

/* ---------------------------- compression ---------------------------- */
typedef struct {
    const sched_t *S;
    const float *x;
    float *xr;
    uint8_t *known;
    uint16_t *codes;
    int radius;
    const float *e, *twoe, *inv2e;
    uint32_t *out_idx;
    float *out_val;
    int64_t capacity;
    int64_t n_out;
    int bad;
} cctx_t;

/* Quantization (Sec. III-A; spec rule q = round((x - p) / 2e)):
 * q = rint((x - p) * inv2e); |q| >= R or a reconstruction outside the bound
 * makes the point an outlier (code 0, x' = x); otherwise code = q + R and
 * x' = p + (float)(code - R) * 2e. */
static void compress_visit(void *vctx, const int64_t c[3], int d, int l)
{
    cctx_t *C = (cctx_t *)vctx;
    int64_t i = lin(C->S, c);
    int kind;
    float p = predict_point(C->S, C->xr, C->known, c, d, l, &kind, &C->bad);
    float xv = C->x[i];
    float diff = xv - p;
    float v = diff * C->inv2e[l];
    float q = rintf(v);
    int outlier = 1;
    if (fabsf(q) < (float)C->radius) {
        int32_t qi = (int32_t)q;
        float xrv = p + (float)qi * C->twoe[l];
        if (fabsf(xv - xrv) <= C->e[l]) {
            C->codes[i] = (uint16_t)(qi + C->radius);
            C->xr[i] = xrv;
            outlier = 0;
        }
    }
    if (outlier) {
        C->codes[i] = 0;
        C->xr[i] = xv;
    }
    C->known[i] = 1;
}

/* Collect outliers in ascending index (stream compaction, Sec. V-A). */
static void collect_outliers(cctx_t *C, int64_t n)
{
    C->n_out = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (C->codes[i] != 0) continue;
        if (C->n_out < C->capacity) {
            C->out_idx[C->n_out] = (uint32_t)i;
            C->out_val[C->n_out] = C->x[i];
        }
        C->n_out++;
    }
}

static void fill_anchors(const sched_t *S, const float *x, float *anchors, float *xr, uint8_t *known,
                         uint16_t *codes, int radius)
{
    const int64_t *A = S->A;
    int64_t ay = anchors_along(S->dims[1], A[1]), ax = anchors_along(S->dims[2], A[2]);
    for (int64_t z = 0; z < S->dims[0]; z += A[0])
        for (int64_t y = 0; y < S->dims[1]; y += A[1])
            for (int64_t xx = 0; xx < S->dims[2]; xx += A[2]) {
                int64_t c[3] = {z, y, xx};
                int64_t i = lin(S, c);
                int64_t a = ((z / A[0]) * ay + y / A[1]) * ax + xx / A[2];
                if (x) anchors[a] = x[i];
                xr[i] = anchors[a];
                if (known) known[i] = 1;
                if (codes) codes[i] = (uint16_t)radius;
            }
}

/* Compress: returns the true outlier count (entries beyond `capacity` are
 * not written), or -1 when a prediction read an undefined value (a broken
 * schedule; cannot happen for a correct one).  xr receives x'. */
int64_t orc_compress(const float *x, int64_t nz, int64_t ny, int64_t nx,
                     const int32_t order[3], const int32_t level_kind[3], const int32_t cubic_kind[3],
                     int32_t domain_x, int32_t ndim, int32_t radius, const float *e, const float *twoe,
                     const float *inv2e, float *anchors, uint16_t *codes, uint32_t *out_idx, float *out_val,
                     int64_t capacity, float *xr)
{
    sched_t S;
    if (sched_init(&S, nz, ny, nx, order, level_kind, cubic_kind, domain_x, ndim)) return -2;
    int64_t n = nz * ny * nx;
    uint8_t *known = (uint8_t *)calloc((size_t)n, 1);
    if (!known) return -3;
    for (int64_t i = 0; i < n; ++i) xr[i] = NAN;
    fill_anchors(&S, x, anchors, xr, known, codes, radius);
    cctx_t C = {&S, x, xr, known, codes, radius, e, twoe, inv2e, out_idx, out_val, capacity, 0, 0};
    for_each_pass(&S, compress_visit, &C);
    for (int64_t i = 0; i < n; ++i)
        if (!known[i]) C.bad = 1;   /* every point must be visited */
    free(known);
    if (C.bad) return -1;
    collect_outliers(&C, n);
    return C.n_out;
}

/* --------------------------- decompression --------------------------- */
typedef struct {
    const sched_t *S;
    const uint16_t *codes;
    float *xr;
    uint8_t *known;
    int radius;
    const float *twoe;
    int bad;
} dctx_t;

static void decompress_visit(void *vctx, const int64_t c[3], int d, int l)
{
    dctx_t *D = (dctx_t *)vctx;
    int64_t i = lin(D->S, c);
    int kind;
    float p = predict_point(D->S, D->xr, D->known, c, d, l, &kind, &D->bad);
    uint16_t code = D->codes[i];
    if (code != 0) {
        int32_t qi = (int32_t)code - D->radius;
        D->xr[i] = p + (float)qi * D->twoe[l];
    }
    /* code 0: xr[i] already holds the outlier's stored value */
    D->known[i] = 1;
}

/* Decompress: replays the compression order (Sec. IV-B.1: decompression
 * replays the prediction from the quant-codes).  Returns 0, or -1 on an
 * undefined read / missing outlier value. */
int orc_decompress(int64_t nz, int64_t ny, int64_t nx,
                   const int32_t order[3], const int32_t level_kind[3], const int32_t cubic_kind[3],
                   int32_t domain_x, int32_t ndim, int32_t radius, const float *twoe,
                   const float *anchors, const uint16_t *codes,
                   const uint32_t *out_idx, const float *out_val, int64_t n_out, float *xr)
{
    sched_t S;
    if (sched_init(&S, nz, ny, nx, order, level_kind, cubic_kind, domain_x, ndim)) return -2;
    int64_t n = nz * ny * nx;
    uint8_t *known = (uint8_t *)calloc((size_t)n, 1);
    if (!known) return -3;
    for (int64_t i = 0; i < n; ++i) xr[i] = NAN;
    fill_anchors(&S, NULL, (float *)anchors, xr, known, NULL, radius);
    uint8_t *has_out = (uint8_t *)calloc((size_t)n, 1);
    for (int64_t j = 0; j < n_out; ++j) {
        xr[out_idx[j]] = out_val[j];
        has_out[out_idx[j]] = 1;
    }
    int bad = 0;
    for (int64_t i = 0; i < n; ++i)
        if (codes[i] == 0 && !has_out[i]) bad = 1;
    free(has_out);
    dctx_t D = {&S, codes, xr, known, radius, twoe, 0};
    for_each_pass(&S, decompress_visit, &D);
    free(known);
    return (bad || D.bad) ? -1 : 0;
}

/* ------------- debug mode: prediction from ORIGINAL neighbours ------------- */
typedef struct {
    const sched_t *S;
    const float *x;
    float *pred;
    uint8_t *kind;
    int bad;
} pctx_t;

static void predict_visit(void *vctx, const int64_t c[3], int d, int l)
{
    pctx_t *P = (pctx_t *)vctx;
    int64_t i = lin(P->S, c);
    int kind;
    P->pred[i] = predict_point(P->S, P->x, NULL, c, d, l, &kind, &P->bad);
    if (P->kind) P->kind[i] = (uint8_t)kind;
}

int orc_predict_original(const float *x, int64_t nz, int64_t ny, int64_t nx,
                         const int32_t order[3], const int32_t level_kind[3],
                         const int32_t cubic_kind[3], int32_t domain_x, int32_t ndim, float *pred, uint8_t *kind)
{
    sched_t S;
    if (sched_init(&S, nz, ny, nx, order, level_kind, cubic_kind, domain_x, ndim)) return -2;
    int64_t n = nz * ny * nx;
    for (int64_t i = 0; i < n; ++i) {
        pred[i] = x[i];
        if (kind) kind[i] = K_ANCHOR;
    }
    pctx_t P = {&S, x, pred, kind, 0};
    for_each_pass(&S, predict_visit, &P);
    return 0;
}

/* ---------------- quant-code histogram (Fig. 1 statistics, Sec. V-A) ---------------- */
void orc_histogram(const uint16_t *codes, int64_t n, int32_t radius, uint32_t *hist)
{
    memset(hist, 0, sizeof(uint32_t) * (size_t)(2 * radius));
    for (int64_t i = 0; i < n; ++i)
        if (codes[i] < 2 * radius) hist[codes[i]]++;
}

/* ------------- sampling profile and auto-tuning (Sec. IV-B.1, IV-B.2) -------------
 * Samples: a 4x4x4 sub-grid, coordinate j along an axis of length n is
 * lo + floor(j * (n - 1 - 2*lo) / 3) with lo = min(12, floor((n-1)/2)).
 * At every sample and along every axis, with neighbours taken from the
 * ORIGINAL values:
 *   prof[3*d + 0]  += |x - NAK cubic (stride 1)|
 *   prof[3*d + 1]  += |x - natural cubic (stride 1)|
 *   prof[9 + d]    += |x - linear (stride 1)|
 *   prof[12 + d]   += 2 |x - linear (stride 2)|
 *   prof[15 + d]   += |x - quad-left (stride 2)| + |x - quad-right (stride 2)|
 * (prof[3*d + 2] is unused).  A test whose neighbours fall outside the field
 * is skipped, and so are the axes that are not chunked (the leading axes of a
 * 1-D or 2-D field).  Sums are in double, in sample order (z, y, x ascending),
 * axis by axis. */
#define ORC_PROF_LEN 18

static int64_t sample_coord(int64_t n, int j)
{
    int64_t lo = (n - 1) / 2;
    if (lo > 12) lo = 12;
    return lo + (int64_t)j * (n - 1 - 2 * lo) / 3;
}

void orc_profile(const float *x, int64_t nz, int64_t ny, int64_t nx, int32_t ndim, double *prof)
{
    int64_t dims[3] = {nz, ny, nx};
    int64_t stride[3] = {ny * nx, nx, 1};
    for (int t = 0; t < ORC_PROF_LEN; ++t) prof[t] = 0.0;
    for (int d = 3 - ndim; d < 3; ++d)
        for (int jz = 0; jz < 4; ++jz)
            for (int jy = 0; jy < 4; ++jy)
                for (int jx = 0; jx < 4; ++jx) {
                    int64_t c[3] = {sample_coord(nz, jz), sample_coord(ny, jy), sample_coord(nx, jx)};
                    int64_t i = (c[0] * ny + c[1]) * nx + c[2];
                    int64_t n = c[d], nd = dims[d], sd = stride[d];
                    double xv = (double)x[i];
                    if (n - 3 >= 0 && n + 3 <= nd - 1) {
                        float m3 = x[i - 3 * sd], m1 = x[i - sd], p1 = x[i + sd], p3 = x[i + 3 * sd];
                        prof[3 * d + 0] += fabs(xv - (double)orc_spline(K_CUBIC_NAK, m3, m1, p1, p3));
                        prof[3 * d + 1] += fabs(xv - (double)orc_spline(K_CUBIC_NATURAL, m3, m1, p1, p3));
                    }
                    if (n - 1 >= 0 && n + 1 <= nd - 1) {
                        float m1 = x[i - sd], p1 = x[i + sd];
                        prof[9 + d] += fabs(xv - (double)orc_spline(K_LINEAR, 0.0f, m1, p1, 0.0f));
                    }
                    if (n - 6 >= 0 && n + 6 <= nd - 1) {
                        float m3 = x[i - 6 * sd], m1 = x[i - 2 * sd], p1 = x[i + 2 * sd], p3 = x[i + 6 * sd];
                        prof[12 + d] += 2.0 * fabs(xv - (double)orc_spline(K_LINEAR, 0.0f, m1, p1, 0.0f));
                        prof[15 + d] += fabs(xv - (double)orc_spline(K_QUAD_LEFT, m3, m1, p1, 0.0f))
                                      + fabs(xv - (double)orc_spline(K_QUAD_RIGHT, 0.0f, m1, p1, p3));
                    }
                }
}

/* Decision (Sec. IV-B.2): per axis the cubic with the lower error (not-a-knot
 * wins ties); axes ordered by descending error of their chosen cubic (ties:
 * lower axis id first); per level, linear iff its error is strictly smaller
 * than the spline's; stride 4 keeps the spline setting (inside an 8^3 chunk
 * every stride-4 stencil is linear or a copy either way). */
void orc_autotune_decide(const double *prof, int32_t order[3], int32_t level_kind[3], int32_t cubic_kind[3])
{
    double err[3];
    for (int d = 0; d < 3; ++d) {
        cubic_kind[d] = (prof[3 * d + 1] < prof[3 * d + 0]) ? 1 : 0;
        err[d] = prof[3 * d + cubic_kind[d]];
    }
    int ord[3] = {0, 1, 2};
    /* stable selection sort by descending err */
    for (int a = 0; a < 3; ++a) {
        int best = a;
        for (int b = a + 1; b < 3; ++b)
            if (err[ord[b]] > err[ord[best]]) best = b;
        int t = ord[best];
        for (int b = best; b > a; --b) ord[b] = ord[b - 1];
        ord[a] = t;
    }
    for (int a = 0; a < 3; ++a) order[a] = ord[a];
    double spline1 = err[0] + err[1] + err[2];
    double lin1 = prof[9] + prof[10] + prof[11];
    double lin2 = prof[12] + prof[13] + prof[14];
    double quad2 = prof[15] + prof[16] + prof[17];
    level_kind[0] = (lin1 < spline1) ? 0 : 1;
    level_kind[1] = (lin2 < quad2) ? 0 : 1;
    level_kind[2] = 1;
}
