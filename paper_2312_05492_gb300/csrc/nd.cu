// 1-D and 2-D G-Interp (Sec. IV-A: 16^2 chunks for 2-D data, 512-point chunks
// for 1-D data), compression and decompression.
//
// Geometry.  A field of dims {nz, ny, nx} is chunked on its last ndim axes with
// anchor stride A (16 or 512) and interpolated at strides A/2, ..., 1 (L = 4 or 9
// levels), one chunked axis at a time in dim order; the leading axes hold
// independent slices (2-D: every z) or rows (1-D: every (z, y)).  Level bounds
// e_l = e / alpha^l (Sec. IV-B.1) for all L levels; levels coarser than stride 4
// use level_kind[2].
//
// Tiles: 2-D tiles own 16 rows x 128 columns of one slice, 1-D tiles 2048 points
// of one row.  Persistent CTAs take tiles in turn; a CTA stages the tile with its
// closing row and column (the anchors and points its chunks borrow from the next
// tile) in shared memory, runs every pass on it, and writes only what it owns.
// Passes inside a tile are separated by barriers; tiles are independent.  2-D passes
// work on chunk lines (the 17 points of one chunk along the pass axis, its known
// points in registers, split in two at the fine strides); 1-D passes of whole tiles
// on segments of 4, 2 or 1 points.  Tiles clipped by the field's end take the
// neighbour-count rule per point.  2-D tiles stage the next tile asynchronously while
// the current one is worked on; whole-width tiles write 8 codes (or 4 values) per
// 16-byte store.
// The level constants (double arithmetic, slow on this part) are formed once per
// CTA, one thread per level.
//
// Outputs match the 3-D path's formats: codes (q + R, 0 for outliers, R at
// anchors), anchors [nz'][ny'][nx'], the fused histogram, and the outlier bitmap
// (one word per 32 x-positions of a row, here in row-major order: a 1-D tile's
// words are contiguous) with per-block popcounts for the ordered compaction.
#include "tma.cuh"

namespace gi {
namespace {

constexpr int ND_THREADS = 256;
constexpr int ND_MAX_LEVELS = 9;
constexpr int ND_HIST_SMEM_BINS = 8192;
// persistent CTAs per SM: 6 for 1-D (registers capped at 40); 5 for 2-D (48 registers:
// with the next tile staged asynchronously, faster than 6 with 40 or 4 with 64)
template <int NDIM>
constexpr int nd_ctas_per_sm() { return NDIM == 2 ? 5 : 6; }

template <int NDIM>
struct NdGeom;
template <>
struct NdGeom<2> {
    static constexpr int A = 16, L = 4;
    static constexpr int TY = 16, TX = 128;    // owned rows x columns
    static constexpr int BY = 17, BX = 129;    // staged box
    static constexpr int PX = 129;             // row pitch (odd: column walks hit distinct banks)
    static constexpr int CPX = 130;            // code-box row pitch (65 words, odd; rows 4-byte aligned)
};
template <>
struct NdGeom<1> {
    static constexpr int A = 512, L = 9;
    static constexpr int TY = 1, TX = 2048;
    static constexpr int BY = 1, BX = 2049;
    static constexpr int PX = 2049;
    static constexpr int CPX = 2050;
};

// Shared-memory index of box element i.  1-D passes walk the row with stride 2s
// (up to 512 words), which would put a warp's accesses in one bank; one pad word
// after every 32 spreads them.  2-D boxes (odd row pitch) are unpadded.
template <int NDIM>
__device__ __forceinline__ int vix(int i) { return NDIM == 1 ? i + (i >> 5) : i; }
// the same for 16-bit arrays: one pad word (two halves) after every 32 words
template <int NDIM>
__device__ __forceinline__ int hix(int j) { return NDIM == 1 ? j + ((j >> 6) << 1) : j; }
template <int NDIM>
__host__ __device__ constexpr int vsize(int n) { return NDIM == 1 ? n + (n >> 5) + 1 : n; }
template <int NDIM>
__host__ __device__ constexpr int hsize(int n) { return NDIM == 1 ? n + ((n >> 6) << 1) + 2 : n; }

// the 16 bits of x moved to the even bit positions (bit i -> bit 2i)
__device__ __forceinline__ uint32_t spread16(uint32_t x)
{
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

struct NdTile {
    long long row0;  // first global (z, y) row of the tile: z * ny + y0
    int z, y0, x0;   // tile origin
    int ey, ex;      // largest local index staged along y and x (box clipped to the field)
    int oy, ox;      // owned rows and columns (clipped to the field)
};

template <int NDIM>
__device__ __forceinline__ NdTile nd_tile(Dims d, int b)
{
    using G = NdGeom<NDIM>;
    const int ntx = (d.nx + G::TX - 1) / G::TX;
    NdTile t;
    const int tx = b % ntx;
    const int r = b / ntx;  // 2-D: z * nty + ty; 1-D: z * ny + y
    if (NDIM == 2) {
        const int nty = (d.ny + G::TY - 1) / G::TY;
        t.z = r / nty;
        t.y0 = (r - t.z * nty) * G::TY;
    } else {
        t.z = r / d.ny;
        t.y0 = r - t.z * d.ny;
    }
    t.x0 = tx * G::TX;
    t.row0 = (long long)t.z * d.ny + t.y0;
    t.ey = NDIM == 2 ? min(G::BY - 1, d.ny - 1 - t.y0) : 0;
    t.ex = min(G::BX - 1, d.nx - 1 - t.x0);
    t.oy = NDIM == 2 ? min(G::TY, d.ny - t.y0) : 1;
    t.ox = min(G::TX, d.nx - t.x0);
    return t;
}

template <int NDIM>
__device__ __forceinline__ int nd_tiles(Dims d)
{
    using G = NdGeom<NDIM>;
    const int ntx = (d.nx + G::TX - 1) / G::TX;
    const int rows = NDIM == 2 ? d.nz * ((d.ny + G::TY - 1) / G::TY) : d.nz * d.ny;
    return rows * ntx;
}

// Level constants for all L levels, from the header's bound and alpha with the
// same double arithmetic as the header's first three levels (alpha^l by repeated
// multiplication).
template <int L>
__device__ void nd_levels(const interp_header *h, LevelQ *lq)
{
    const int l = threadIdx.x;
    if (l >= L) return;
    double apow = 1.0;
    for (int j = 0; j < l; ++j) apow *= h->alpha;
    const float e = (float)(h->eb_abs / apow);
    lq[l] = LevelQ{e, 2.0f * e, (float)(1.0 / (2.0 * (double)e))};
}

struct NdPass {
    int a;       // interpolation axis: 1 = y, 2 = x
    int na, no;  // points along the axis and along the other axis
    int so;      // step along the other axis (s or 2s)
    int ea;      // largest staged local index along the axis
    int sa;      // shared-memory stride along the axis
    int so_mem;  // shared-memory stride along the other axis
};

// Stencil by the neighbour count within the closed chunk [lo, lo + A] (clipped to
// the staged box, whose end is the field's end or the chunk's closing point),
// Sec. IV-B.1: 4 neighbours cubic, 3 quadratic, 2 linear, 1 copy of x_{n-s}.
template <int NDIM>
__device__ __forceinline__ float nd_predict(const float *v, int i, int n, int s, int ea, int sa, int spline,
                                           const Cubic &ck)
{
    constexpr int A = NdGeom<NDIM>::A;
    const int lo = (n / A) * A;
    const int hi = min(lo + A, ea);
    const float m1 = v[vix<NDIM>(i - s * sa)];
    if (n + s > hi) return m1;
    const float p1 = v[vix<NDIM>(i + s * sa)];
    if (!spline) return sp_linear(m1, p1);
    const bool has_m3 = n - 3 * s >= lo, has_p3 = n + 3 * s <= hi;
    if (has_m3 && has_p3) return sp_cubic(ck, v[vix<NDIM>(i - 3 * s * sa)], m1, p1, v[vix<NDIM>(i + 3 * s * sa)]);
    if (has_m3) return sp_quad_left(v[vix<NDIM>(i - 3 * s * sa)], m1, p1);
    if (has_p3) return sp_quad_right(m1, p1, v[vix<NDIM>(i + 3 * s * sa)]);
    return sp_linear(m1, p1);
}

template <int NDIM>
__device__ __forceinline__ NdPass nd_pass(const NdTile &t, const int order[3], int k, int s)
{
    using G = NdGeom<NDIM>;
    NdPass p;
    p.a = order[k];
    if (NDIM == 1) {
        p.ea = t.ex;
        p.sa = 1;
        p.no = 1;
        p.so = 1;
        p.so_mem = 0;
    } else {
        const int o = p.a == 1 ? 2 : 1;
        int ko = 0;
        for (int j = 0; j < 3; ++j)
            if (order[j] == o) ko = j;
        p.so = ko < k ? s : 2 * s;
        const int eo = o == 1 ? t.ey : t.ex;
        p.no = eo / p.so + 1;
        p.ea = p.a == 1 ? t.ey : t.ex;
        p.sa = p.a == 1 ? G::PX : 1;
        p.so_mem = o == 1 ? G::PX : 1;
    }
    p.na = p.ea >= s ? (p.ea - s) / (2 * s) + 1 : 0;
    return p;
}

// Configuration from the header: order with the chunked axes, level kinds, cubics.
struct NdCfg {
    int order[3];
    int level_kind[3];
    int cubic_kind[3];
};

__device__ __forceinline__ NdCfg nd_cfg(const interp_header *h)
{
    NdCfg c;
    for (int j = 0; j < 3; ++j) {
        c.order[j] = h->cfg.dim_order[j];
        c.level_kind[j] = h->cfg.level_kind[j];
        c.cubic_kind[j] = h->cfg.cubic_kind[j];
    }
    return c;
}

// Stage a full box (BY x BX elements, row pitch PX in shared memory) with every
// thread's loads issued before any of them is stored: the box is one flat index
// space split over the threads, ceil(BY*BX / ND_THREADS) loads each.
template <int NDIM, typename T>
__device__ __forceinline__ void nd_stage_full(T *dst, const T *src, long long row0, int nx, int x0)
{
    using G = NdGeom<NDIM>;
    constexpr int NE = G::BY * G::BX;
    constexpr int K = (NE + ND_THREADS - 1) / ND_THREADS;
    T r[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = threadIdx.x + k * ND_THREADS;
        if (e < NE) {
            const int by = e / G::BX, bx = e - by * G::BX;
            r[k] = __ldg(src + (row0 + by) * nx + x0 + bx);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = threadIdx.x + k * ND_THREADS;
        if (e < NE) {
            const int by = e / G::BX, bx = e - by * G::BX;
            const int j = by * (sizeof(T) == 4 ? G::PX : G::CPX) + bx;
            dst[sizeof(T) == 4 ? vix<NDIM>(j) : hix<NDIM>(j)] = r[k];
        }
    }
}

// ---- full tiles: the staged box lies inside the field, so every chunk is whole
// and every pass has a shape known at compile time (no runtime division, and the
// stencil depends only on the point's position in its chunk).
struct NdPointCtx {
    LevelQ q;
    Cubic ck;
    int spline;
    uint32_t cbias;
    float Rf;
    uint16_t *cs;          // compression: owned codes [TY][TX]
    const uint16_t *cb;    // decompression: the box's codes
    const float *xrec;     // decompression: outlier values (scattered beforehand)
    long long row0;
    int nx, x0;
};

template <int NDIM, int S, int AX, int SO, bool COMPRESS>
__device__ __forceinline__ void nd_full_pass(float *v, const NdPointCtx &c)
{
    using G = NdGeom<NDIM>;
    constexpr int A = G::A;
    constexpr int EA = AX == 1 ? G::BY - 1 : G::BX - 1;
    constexpr int EO = NDIM == 1 ? 0 : (AX == 1 ? G::BX - 1 : G::BY - 1);
    constexpr int NA = (EA - S) / (2 * S) + 1;
    constexpr int NO = EO / SO + 1;
    constexpr int SA = AX == 1 ? G::PX : 1;
    constexpr int SOM = AX == 1 ? 1 : G::PX;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < NA * NO; idx += ND_THREADS) {
        int ia, io;
        if (AX == 2) {
            ia = idx % NA;
            io = idx / NA;
        } else {
            io = idx % NO;
            ia = idx / NO;
        }
        const int n = S + 2 * S * ia, m = io * SO;
        const int i = n * SA + m * SOM;
        const int r = n % A;  // chunk [n - r, n - r + A], whole: x_{n+s} always exists
        const float m1 = v[vix<NDIM>(i - S * SA)], p1 = v[vix<NDIM>(i + S * SA)];
        float pred;
        if (!c.spline) {
            pred = sp_linear(m1, p1);
        } else {
            const bool hm3 = r >= 3 * S, hp3 = r + 3 * S <= A;
            if (hm3 && hp3) pred = sp_cubic(c.ck, v[vix<NDIM>(i - 3 * S * SA)], m1, p1, v[vix<NDIM>(i + 3 * S * SA)]);
            else if (hm3) pred = sp_quad_left(v[vix<NDIM>(i - 3 * S * SA)], m1, p1);
            else if (hp3) pred = sp_quad_right(m1, p1, v[vix<NDIM>(i + 3 * S * SA)]);
            else pred = sp_linear(m1, p1);
        }
        const int by = AX == 1 ? n : (NDIM == 2 ? m : 0);
        const int bx = AX == 2 ? n : m;
        if (COMPRESS) {
            float xr;
            const int vi = vix<NDIM>(i);
            const uint32_t code = quantize(v[vi], pred, c.q, c.cbias, c.Rf, xr);
            v[vi] = xr;
            if (by < G::TY && bx < G::TX) c.cs[hix<NDIM>(by * G::TX + bx)] = (uint16_t)code;
        } else {
            const uint32_t code = c.cb[hix<NDIM>(i)];
            v[vix<NDIM>(i)] = code ? pred + code_to_q(code, c.cbias) * c.q.twoe
                                   : c.xrec[(c.row0 + by) * c.nx + c.x0 + bx];
        }
    }
}

// Issue the 4-byte asynchronous copies of a tile's value box (the whole box, or the
// part inside the field for a clipped tile) into dst; the copies land while the
// CTA works on the previous tile and are waited for before this one starts.
template <int NDIM>
__device__ __forceinline__ void nd_stage_async(float *dst, const float *src, const NdTile &t, int nx)
{
    using G = NdGeom<NDIM>;
    if (t.ey == G::BY - 1 && t.ex == G::BX - 1) {
        constexpr int NE = G::BY * G::BX;
#pragma unroll 3
        for (int e = threadIdx.x; e < NE; e += ND_THREADS) {
            const int by = e / G::BX, bx = e - by * G::BX;
            cp_async4(dst + vix<NDIM>(by * G::PX + bx), src + (t.row0 + by) * nx + t.x0 + bx);
        }
    } else {
        const int w = t.ex + 1, ne = (t.ey + 1) * w;
        for (int e = threadIdx.x; e < ne; e += ND_THREADS) {
            const int by = e / w, bx = e - by * w;
            cp_async4(dst + vix<NDIM>(by * G::PX + bx), src + (t.row0 + by) * nx + t.x0 + bx);
        }
    }
    cp_async_commit();
}

// Issue the asynchronous copies of a tile's code box, two codes (4 bytes) per copy;
// the field's rows must start on 4-byte boundaries (nx even, codes 4-byte aligned).
// A row's last code whose pair would reach past the field's end is copied alone.
template <int NDIM>
__device__ __forceinline__ void nd_stage_codes_async(uint16_t *dst, const uint16_t *src, const NdTile &t, int nx)
{
    using G = NdGeom<NDIM>;
    auto one = [&](int by, int bx) {
        const uint16_t *sp = src + (t.row0 + by) * nx + t.x0 + bx;
        uint16_t *dp = dst + hix<NDIM>(by * G::CPX + bx);
        if (t.x0 + bx + 1 < nx) cp_async4(dp, sp);
        else *dp = __ldg(sp);
    };
    if (t.ey == G::BY - 1 && t.ex == G::BX - 1) {
        constexpr int NP = (G::BX + 1) / 2;  // pairs per row
#pragma unroll 3
        for (int e = threadIdx.x; e < G::BY * NP; e += ND_THREADS) {
            const int by = e / NP;
            one(by, 2 * (e - by * NP));
        }
    } else {
        const int np = (t.ex + 2) / 2, ne = (t.ey + 1) * np;
        for (int e = threadIdx.x; e < ne; e += ND_THREADS) {
            const int by = e / np;
            one(by, 2 * (e - by * np));
        }
    }
    cp_async_commit();
}

// The anchors a tile's box holds (its own and the closing row and column): thread k
// fetches the k-th into a register, to be stored into the value box at vi.
template <int NDIM>
__device__ __forceinline__ bool nd_anchor_fetch(const float *anchors, Dims d, const NdTile &t, float &val, int &vi)
{
    using G = NdGeom<NDIM>;
    constexpr int NAX = (G::BX - 1) / G::A + 1, NAY = NDIM == 2 ? (G::BY - 1) / G::A + 1 : 1;
    const int k = threadIdx.x;
    if (k >= NAY * NAX) return false;
    const int by = (k / NAX) * G::A, bx = (k % NAX) * G::A;  // y0 is a multiple of A: these rows hold anchors
    if (by > t.ey || bx > t.ex) return false;
    const int ax = (d.nx - 1) / G::A + 1;
    const long long arow = NDIM == 2 ? (long long)t.z * ((d.ny - 1) / G::A + 1) + (t.y0 + by) / G::A : t.row0;
    val = __ldg(anchors + arow * ax + (t.x0 + bx) / G::A);
    vi = vix<NDIM>(by * G::PX + bx);
    return true;
}

// Stage a box clipped by the field's far end ((ey + 1) x (ex + 1) elements) with
// every thread's loads issued before any is stored.
template <int NDIM, typename T>
__device__ __forceinline__ void nd_stage_clipped(T *dst, const T *src, long long row0, int nx, int x0, int ey,
                                                 int ex)
{
    using G = NdGeom<NDIM>;
    constexpr int K = (G::BY * G::BX + ND_THREADS - 1) / ND_THREADS;
    const int w = ex + 1, ne = (ey + 1) * w;
    T r[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = threadIdx.x + k * ND_THREADS;
        if (e < ne) {
            const int by = e / w, bx = e - by * w;
            r[k] = __ldg(src + (row0 + by) * nx + x0 + bx);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = threadIdx.x + k * ND_THREADS;
        if (e < ne) {
            const int by = e / w, bx = e - by * w;
            const int j = by * (sizeof(T) == 4 ? G::PX : G::CPX) + bx;
            dst[sizeof(T) == 4 ? vix<NDIM>(j) : hix<NDIM>(j)] = r[k];
        }
    }
}

// 2-D tiles clipped by the field's far end: chunk segments as for whole tiles, each
// chunk line ending at min(lo + 16, the last staged index) and every point's stencil
// by the neighbour-count rule (Sec. IV-B.1).
template <int S, int AX, bool COMPRESS>
__device__ __forceinline__ void nd2_seg_pass_clipped(float *v, const NdPointCtx &c, int so, int ea, int eo)
{
    using G = NdGeom<2>;
    constexpr int SA = AX == 1 ? G::PX : 1;
    constexpr int SOM = AX == 1 ? 1 : G::PX;
    constexpr int NKMAX = 16 / (2 * S) + 1;
    const int no = eo / so + 1;
    const int nch = ea > 0 ? (ea - 1) / G::A + 1 : 0;  // chunks holding points to predict
#pragma unroll 1
    for (int w = threadIdx.x; w < no * nch; w += ND_THREADS) {
        const int io = w % no, ch = w / no;
        const int m = io * so, n0 = ch * G::A;
        const int hl = min(G::A, ea - n0);  // last offset of the (possibly truncated) chunk line
        float *line = v + m * SOM + n0 * SA;
        float k[NKMAX];
#pragma unroll
        for (int q = 0; q < NKMAX; ++q) k[q] = (2 * q * S <= hl) ? line[q * 2 * S * SA] : 0.0f;
#pragma unroll
        for (int q = 0; q + 1 < NKMAX; ++q) {
            const int o = (2 * q + 1) * S;
            if (o > hl) break;
            float p;
            if (o + S > hl) {
                p = k[q];  // one neighbour: copy of x_{n-s}
            } else if (!c.spline) {
                p = sp_linear(k[q], k[q + 1]);
            } else {
                const bool hm3 = q >= 1, hp3 = o + 3 * S <= hl;
                const float m3 = k[q > 0 ? q - 1 : 0], p3 = k[q + 2 < NKMAX ? q + 2 : q];
                if (hm3 && hp3) p = sp_cubic(c.ck, m3, k[q], k[q + 1], p3);
                else if (hm3) p = sp_quad_left(m3, k[q], k[q + 1]);
                else if (hp3) p = sp_quad_right(k[q], k[q + 1], p3);
                else p = sp_linear(k[q], k[q + 1]);
            }
            const int by = AX == 1 ? n0 + o : m, bx = AX == 2 ? n0 + o : m;
            if (COMPRESS) {
                float xr;
                const uint32_t code = quantize(line[o * SA], p, c.q, c.cbias, c.Rf, xr);
                line[o * SA] = xr;
                if (by < G::TY && bx < G::TX) c.cs[by * G::TX + bx] = (uint16_t)code;
            } else {
                const uint32_t code = c.cb[by * G::CPX + bx];
                line[o * SA] = code ? p + code_to_q(code, c.cbias) * c.q.twoe
                                    : c.xrec[(c.row0 + by) * c.nx + c.x0 + bx];
            }
        }
    }
}

template <int S, bool XFIRST, bool COMPRESS>
__device__ __forceinline__ void nd2_levels_clipped(float *v, NdPointCtx &c, const LevelQ *lq, const NdCfg &cfg,
                                                   int ey, int ex)
{
    constexpr int l = S >= 8 ? 3 : S >= 4 ? 2 : S >= 2 ? 1 : 0;
    c.q = lq[l];
    c.spline = cfg.level_kind[l < 2 ? l : 2];
    constexpr int F = XFIRST ? 2 : 1, O = XFIRST ? 1 : 2;
    c.ck = cubic_coeffs(cfg.cubic_kind[F]);
    nd2_seg_pass_clipped<S, F, COMPRESS>(v, c, 2 * S, F == 2 ? ex : ey, F == 2 ? ey : ex);
    __syncthreads();
    c.ck = cubic_coeffs(cfg.cubic_kind[O]);
    nd2_seg_pass_clipped<S, O, COMPRESS>(v, c, S, O == 2 ? ex : ey, O == 2 ? ey : ex);
    __syncthreads();
    if constexpr (S > 1) nd2_levels_clipped<S / 2, XFIRST, COMPRESS>(v, c, lq, cfg, ey, ex);
}

template <bool COMPRESS>
__device__ __forceinline__ void nd2_clipped_tile(float *v, NdPointCtx &c, const LevelQ *lq, const NdCfg &cfg,
                                                 int ey, int ex)
{
    int px = 0, py = 0;
    for (int j = 0; j < 3; ++j) {
        if (cfg.order[j] == 2) px = j;
        if (cfg.order[j] == 1) py = j;
    }
    if (py < px)
        nd2_levels_clipped<NdGeom<2>::A / 2, false, COMPRESS>(v, c, lq, cfg, ey, ex);
    else
        nd2_levels_clipped<NdGeom<2>::A / 2, true, COMPRESS>(v, c, lq, cfg, ey, ex);
}

// 2-D whole tiles, chunk segments: one work unit is the line of one 16-point chunk
// along the pass axis (its 17 points, the chunk's closing point included); the
// known points (even multiples of s) are loaded once and give all the chunk line's
// predictions from registers, with the stencils of whole chunks (Fig. 3 at twice the
// scale: the first point right-quadratic, the last left-quadratic, the rest cubic;
// a lone midpoint linear).
// Pieces per chunk line of a whole-tile pass at stride S: two at the fine strides,
// where a line holds 4 or 8 predictions, so that more threads work (2-D compression
// 0.858 -> 0.839 ms on 32 x 2048^2; decompression unchanged).
__host__ __device__ constexpr int nd2_pieces(int S, int /*AX*/) { return S <= 2 ? 2 : 1; }

// A chunk line may be split into H pieces of (NK - 1) / H predictions each (more
// work units, shorter chains); a piece also loads the known points just outside it
// that its cubic stencils need.
template <int S, int AX, int SO, bool COMPRESS, int H = 1>
__device__ __forceinline__ void nd2_seg_pass(float *v, const NdPointCtx &c)
{
    using G = NdGeom<2>;
    constexpr int NO = (AX == 2 ? G::BY - 1 : G::BX - 1) / SO + 1;  // lines along the other axis
    constexpr int NCH = AX == 2 ? G::TX / G::A : 1;                 // chunks along the axis
    constexpr int SA = AX == 1 ? G::PX : 1;
    constexpr int SOM = AX == 1 ? 1 : G::PX;
    constexpr int NK = 16 / (2 * S) + 1;  // known points of a chunk line
    constexpr int NPH = (NK - 1) / H;     // predictions per piece
    static_assert(NPH * H == NK - 1 && (H == 1 || NPH >= 2), "pieces split a chunk line evenly");
#pragma unroll 1
    for (int w = threadIdx.x; w < NO * NCH * H; w += ND_THREADS) {
        const int io = w % NO, r = w / NO;  // consecutive threads take consecutive lines
        const int h = H == 1 ? 0 : r % H, ch = H == 1 ? r : r / H;
        const int m = io * SO, n0 = ch * G::A;
        float *line = v + m * SOM + n0 * SA;
        const int q0 = h * NPH;  // the piece's first prediction
        // kk[j] = known point q0 - 1 + j of the chunk line (outside the line: unused)
        float kk[NPH + 3];
#pragma unroll
        for (int j = 0; j < NPH + 3; ++j) {
            const int q = q0 - 1 + j;
            kk[j] = (H == 1 && (j == 0 || j == NPH + 2)) ? 0.0f
                    : (q >= 0 && q < NK) ? line[q * 2 * S * SA] : 0.0f;
        }
        auto emit = [&](int q, float p) {  // prediction of the point between known q and q + 1
            const int o = (2 * q + 1) * S;
            const int by = AX == 1 ? n0 + o : m, bx = AX == 2 ? n0 + o : m;
            if (COMPRESS) {
                float xr;
                const uint32_t code = quantize(line[o * SA], p, c.q, c.cbias, c.Rf, xr);
                line[o * SA] = xr;
                if (by < G::TY && bx < G::TX) c.cs[by * G::TX + bx] = (uint16_t)code;
            } else {
                const uint32_t code = c.cb[by * G::CPX + bx];
                line[o * SA] = code ? p + code_to_q(code, c.cbias) * c.q.twoe
                                    : c.xrec[(c.row0 + by) * c.nx + c.x0 + bx];
            }
        };
        if (!c.spline || NK == 2) {
#pragma unroll
            for (int j = 1; j <= NPH; ++j) emit(q0 + j - 1, sp_linear(kk[j], kk[j + 1]));
        } else {
#pragma unroll
            for (int j = 1; j <= NPH; ++j) {
                const int q = q0 + j - 1;
                float p;
                if (q == 0) p = sp_quad_right(kk[j], kk[j + 1], kk[j + 2]);
                else if (q == NK - 2) p = sp_quad_left(kk[j - 1], kk[j], kk[j + 1]);
                else p = sp_cubic(c.ck, kk[j - 1], kk[j], kk[j + 1], kk[j + 2]);
                emit(q, p);
            }
        }
    }
}

// 1-D whole tiles, segments: one work unit is P consecutive points of a level-S pass
// (P = 4 at stride 1, 2 at stride 2, else 1), whose known neighbours at even multiples
// of S give all its predictions from registers, plus the known points just outside
// the segment where the segment does not start or end a chunk.  Every chunk is whole:
// the first point of a chunk has no x_{n-3s} (right quadratic), the last no x_{n+3s}
// (left quadratic), a lone midpoint neither (linear), the rest are cubic (Sec. IV-B.1).
template <int S, bool COMPRESS>
__device__ __forceinline__ void nd1_seg_pass(float *v, const NdPointCtx &c)
{
    using G = NdGeom<1>;
    constexpr int A = G::A;
    // points per segment: as many as keep one segment per thread (NSEG >= ND_THREADS)
    constexpr int P = S == 1 ? 4 : (S == 2 ? 2 : 1);
    constexpr int SPAN = 2 * S * P;                           // the segment's known points: 0, 2S, .., SPAN
    constexpr int NSEG = G::TX / SPAN;
#pragma unroll 1
    for (int w = threadIdx.x; w < NSEG; w += ND_THREADS) {
        const int n0 = w * SPAN;
        const bool at_lo = n0 % A == 0, at_hi = (n0 + SPAN) % A == 0;  // the segment starts / ends a chunk
        float k[P + 3];  // k[q + 1] = x_{n0 + 2Sq}, q = -1 .. P + 1
#pragma unroll
        for (int q = 0; q <= P; ++q) k[q + 1] = v[vix<1>(n0 + 2 * S * q)];
        k[0] = 0.0f;
        k[P + 2] = 0.0f;
        if (c.spline) {
            if (!at_lo) k[0] = v[vix<1>(n0 - 2 * S)];
            if (!at_hi) k[P + 2] = v[vix<1>(n0 + SPAN + 2 * S)];
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int o = n0 + (2 * q + 1) * S;
            const float m1 = k[q + 1], p1 = k[q + 2];
            float p;
            if (!c.spline) {
                p = sp_linear(m1, p1);
            } else {
                const bool hm3 = q > 0 || !at_lo, hp3 = q < P - 1 || !at_hi;
                if (hm3 && hp3) p = sp_cubic(c.ck, k[q], m1, p1, k[q + 3]);
                else if (hm3) p = sp_quad_left(k[q], m1, p1);
                else if (hp3) p = sp_quad_right(m1, p1, k[q + 3]);
                else p = sp_linear(m1, p1);
            }
            if (COMPRESS) {
                float xr;
                const int vi = vix<1>(o);
                const uint32_t code = quantize(v[vi], p, c.q, c.cbias, c.Rf, xr);
                v[vi] = xr;
                c.cs[hix<1>(o)] = (uint16_t)code;
            } else {
                const uint32_t code = c.cb[hix<1>(o)];
                v[vix<1>(o)] = code ? p + code_to_q(code, c.cbias) * c.q.twoe : c.xrec[c.row0 * c.nx + c.x0 + o];
            }
        }
    }
}

// Levels S, S/2, ..., 1 of a full tile; in 2-D the axis interpolated first in a level
// sees the other on the 2s-grid, the second on the s-grid.
template <int NDIM, int S, bool XFIRST, bool COMPRESS>
__device__ __forceinline__ void nd_full_levels(float *v, NdPointCtx &c, const LevelQ *lq, const NdCfg &cfg)
{
    constexpr int l = S >= 256 ? 8 : S >= 128 ? 7 : S >= 64 ? 6 : S >= 32 ? 5 : S >= 16 ? 4 : S >= 8 ? 3 : S >= 4 ? 2
                                                                                                            : S >= 2 ? 1 : 0;
    c.q = lq[l];
    c.spline = cfg.level_kind[l < 2 ? l : 2];
    if (NDIM == 1) {
        c.ck = cubic_coeffs(cfg.cubic_kind[2]);
        nd1_seg_pass<S, COMPRESS>(v, c);
        __syncthreads();
    } else {
        constexpr int F = XFIRST ? 2 : 1, O = XFIRST ? 1 : 2;
        c.ck = cubic_coeffs(cfg.cubic_kind[F]);
        nd2_seg_pass<S, F, 2 * S, COMPRESS, nd2_pieces(S, F)>(v, c);
        __syncthreads();
        c.ck = cubic_coeffs(cfg.cubic_kind[O]);
        nd2_seg_pass<S, O, S, COMPRESS, nd2_pieces(S, O)>(v, c);
        __syncthreads();
    }
    if constexpr (S > 1) nd_full_levels<NDIM, S / 2, XFIRST, COMPRESS>(v, c, lq, cfg);
}

template <int NDIM, bool COMPRESS>
__device__ __forceinline__ void nd_full_tile(float *v, NdPointCtx &c, const LevelQ *lq, const NdCfg &cfg)
{
    using G = NdGeom<NDIM>;
    int px = 0, py = 0;
    for (int j = 0; j < 3; ++j) {
        if (cfg.order[j] == 2) px = j;
        if (cfg.order[j] == 1) py = j;
    }
    if (NDIM == 2 && py < px)
        nd_full_levels<NDIM, G::A / 2, false, COMPRESS>(v, c, lq, cfg);
    else
        nd_full_levels<NDIM, G::A / 2, true, COMPRESS>(v, c, lq, cfg);
}

template <int NDIM>
__device__ __forceinline__ void nd_compress_tile(const CompressArgs &a, const NdCfg &cfg, const LevelQ *lq, float *v,
                                                 uint16_t *cs, uint32_t *hs, bool smem_hist, uint32_t &central,
                                                 int b)
{
    using G = NdGeom<NDIM>;
    constexpr int L = G::L;
    const Dims d = a.dims;
    const int tid = threadIdx.x;
    const int bins = 2 * a.radius;
    const uint32_t cbias = kMagicBits - (uint32_t)a.radius;
    const float Rf = (float)a.radius;
    const NdTile t = nd_tile<NDIM>(d, b);

    // the box was staged by nd_stage_async (landed and visible: the caller waited)
    const bool full = t.ey == G::BY - 1 && t.ex == G::BX - 1;
    // owned anchors: code R, value kept
    for (int i = tid; i < hsize<NDIM>(G::TY * G::TX); i += ND_THREADS) cs[i] = (uint16_t)a.radius;
    __syncthreads();

    if (full || NDIM == 2) {
        NdPointCtx c;
        c.cbias = cbias;
        c.Rf = Rf;
        c.cs = cs;
        if (full) nd_full_tile<NDIM, true>(v, c, lq, cfg);
        else nd2_clipped_tile<true>(v, c, lq, cfg, t.ey, t.ex);
    }
    for (int l = (full || NDIM == 2) ? -1 : L - 1; l >= 0; --l) {
        const int s = 1 << l;
        const LevelQ q = lq[l];
        const int spline = cfg.level_kind[l < 2 ? l : 2];
        for (int k = 0; k < 3; ++k) {
            if (cfg.order[k] < 3 - NDIM) continue;  // not a chunked axis
            const NdPass p = nd_pass<NDIM>(t, cfg.order, k, s);
            const Cubic ck = cubic_coeffs(cfg.cubic_kind[p.a]);
            const int npts = p.na * p.no;
            for (int idx = tid; idx < npts; idx += ND_THREADS) {
                // consecutive threads walk x: along the axis for x-passes, along the other axis for y-passes
                int ia, io;
                if (p.a == 2) {
                    ia = idx % p.na;
                    io = idx / p.na;
                } else {
                    io = idx % p.no;
                    ia = idx / p.no;
                }
                const int n = s + 2 * s * ia, m = io * p.so;
                const int i = n * p.sa + m * p.so_mem;
                const float pred = nd_predict<NDIM>(v, i, n, s, p.ea, p.sa, spline, ck);
                float xr;
                const uint32_t code = quantize(v[vix<NDIM>(i)], pred, q, cbias, Rf, xr);
                v[vix<NDIM>(i)] = xr;
                const int by = p.a == 1 ? n : (NDIM == 2 ? m : 0);
                const int bx = p.a == 2 ? n : m;
                if (by < G::TY && bx < G::TX) cs[hix<NDIM>(by * G::TX + bx)] = (uint16_t)code;
            }
            __syncthreads();
        }
    }

    // owned anchors to the anchor array
    {
        const int ax = (d.nx - 1) / G::A + 1;
        const long long arow = NDIM == 2 ? (long long)t.z * ((d.ny - 1) / G::A + 1) + t.y0 / G::A : t.row0;
        if (t.y0 % G::A == 0 || NDIM == 1)
            for (int bx = tid * G::A; bx < t.ox; bx += ND_THREADS * G::A)
                a.anchors[arow * ax + (t.x0 + bx) / G::A] = v[vix<NDIM>(bx)];
    }

    // codes, outlier bitmap words and the histogram of the owned points
    const int lane = tid & 31, warp = tid >> 5;
    const int wpr = (d.nx + 31) / 32;
    const bool octets = t.ox == G::TX && (d.nx & 7) == 0 && (reinterpret_cast<uintptr_t>(a.codes) & 15u) == 0;
    if (octets) {
        // tiles owning all TX columns, rows 16-byte aligned: a thread takes 8 consecutive
        // codes of a row (one 16-byte load and store); the 4 lanes of a 32-code strip
        // assemble its outlier word, and one atomic per warp carries the block counts
        constexpr int OPR = G::TX / 8;  // octets per row
        const uint32_t R = (uint32_t)a.radius;
        for (int o0 = warp * 32; o0 < G::TY * OPR; o0 += ND_THREADS) {
            const int o = o0 + lane;
            const int by = o / OPR, x8 = 8 * (o - by * OPR);
            const bool in = by < t.oy;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            uint32_t zmask = 0u;
            const long long row = t.row0 + by;
            if (in) {
                const uint32_t *c32 = reinterpret_cast<const uint32_t *>(cs) + hix<NDIM>(by * G::TX + x8) / 2;
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = c32[j];
                *reinterpret_cast<uint4 *>(a.codes + row * d.nx + t.x0 + x8) = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t code = (w[j >> 1] >> (16 * (j & 1))) & 0xffffu;
                    zmask |= (code == 0u ? 1u : 0u) << j;
                    if (a.hist) {
                        if (code == R) ++central;
                        else if (code < (uint32_t)bins) {
                            if (smem_hist) atomicAdd(&hs[code], 1u);
                            else atomicAdd(&a.hist[code], 1u);
                        }
                    }
                }
            }
            uint32_t word = zmask << (8 * (lane & 3));
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            const long long gw = row * wpr + ((t.x0 + x8) >> 5);  // row-major bitmap
            if (in && (lane & 3) == 0) a.bitmap[gw] = word;
            const bool has = in && (lane & 3) == 0 && word != 0u;
            const uint32_t hm = __ballot_sync(0xffffffffu, has);
            if (hm) {
                const long long blk = gw / BITMAP_BLOCK_WORDS;
                const int first = __ffs(hm) - 1;
                const long long b0 = __shfl_sync(0xffffffffu, blk, first);
                uint32_t c = has ? (uint32_t)__popc(word) : 0u;
                if (__all_sync(0xffffffffu, !has || blk == b0)) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
                    if (lane == first) atomicAdd(a.blockcnt + b0, c);
                } else if (has) {
                    atomicAdd(a.blockcnt + blk, c);
                }
            }
        }
        __syncthreads();  // the box and the code stage are reused by the next tile
        return;
    }
    const bool pairs = NDIM == 2 && t.ox == G::TX && (d.nx & 1) == 0 &&
                       (reinterpret_cast<uintptr_t>(a.codes) & 3u) == 0;
    if (pairs) {
        // 2-D tiles owning all 128 columns: a warp step takes 64 codes of a row, two per
        // lane (4-byte loads and stores); the two 32-column words interleave the ballots
        // of the pairs' low and high codes
        const uint32_t *cs2 = reinterpret_cast<const uint32_t *>(cs);
        for (int u = warp; u < t.oy * 2; u += ND_THREADS / 32) {
            const int by = u >> 1, half = u & 1;
            const int c0 = half * 64 + 2 * lane;
            const uint32_t w = cs2[(by * G::TX + c0) >> 1];
            const uint32_t lo = w & 0xffffu, hi = w >> 16;
            const long long row = t.row0 + by;
            *reinterpret_cast<uint32_t *>(a.codes + row * d.nx + t.x0 + c0) = w;
            const uint32_t zl = __ballot_sync(0xffffffffu, lo == 0u), zh = __ballot_sync(0xffffffffu, hi == 0u);
            if (lane == 0) {
                const long long gw = row * wpr + (t.x0 >> 5) + 2 * half;  // row-major bitmap
                const uint32_t w0 = spread16(zl & 0xffffu) | (spread16(zh & 0xffffu) << 1);
                const uint32_t w1 = spread16(zl >> 16) | (spread16(zh >> 16) << 1);
                a.bitmap[gw] = w0;
                a.bitmap[gw + 1] = w1;
                if (w0) atomicAdd(a.blockcnt + gw / BITMAP_BLOCK_WORDS, (uint32_t)__popc(w0));
                if (w1) atomicAdd(a.blockcnt + (gw + 1) / BITMAP_BLOCK_WORDS, (uint32_t)__popc(w1));
            }
            if (a.hist) {
                if (lo == (uint32_t)a.radius) ++central;
                else if (lo < (uint32_t)bins) atomicAdd(smem_hist ? &hs[lo] : &a.hist[lo], 1u);
                if (hi == (uint32_t)a.radius) ++central;
                else if (hi < (uint32_t)bins) atomicAdd(smem_hist ? &hs[hi] : &a.hist[hi], 1u);
            }
        }
        __syncthreads();  // the box and the code stage are reused by the next tile
        return;
    }
    // one 32-column strip of a row per warp step
    const int strips = (t.ox + 31) / 32;
    for (int u = warp; u < t.oy * strips; u += ND_THREADS / 32) {
        const int by = u / strips, strip = u - by * strips, bx = strip * 32 + lane;
        const bool in = bx < t.ox;
        const uint32_t code = in ? cs[hix<NDIM>(by * G::TX + bx)] : 1u;
        const long long row = t.row0 + by;
        if (in) a.codes[row * d.nx + t.x0 + bx] = (uint16_t)code;
        const uint32_t word = __ballot_sync(0xffffffffu, code == 0u);
        if (lane == 0) {
            const long long gw = row * wpr + (t.x0 >> 5) + strip;  // row-major bitmap
            a.bitmap[gw] = word;
            if (word) atomicAdd(a.blockcnt + gw / BITMAP_BLOCK_WORDS, (uint32_t)__popc(word));
        }
        if (a.hist && in) {
            if (code == (uint32_t)a.radius) ++central;
            else if (code < (uint32_t)bins) atomicAdd(smem_hist ? &hs[code] : &a.hist[code], 1u);
        }
    }
    __syncthreads();  // the box and the code stage are reused by the next tile
}

// Asynchronous staging of the next tile pays in 2-D (compression 1.34 -> 1.18 ms,
// decompression 1.13 -> 0.81 ms on 32 x 2048^2); 1-D tiles, whose rows are loaded as
// plain coalesced runs, were slower with it (0.63 -> 0.69 ms decompression) and load
// at each tile's start.
template <int NDIM>
__host__ __device__ constexpr bool nd_async_stage() { return NDIM == 2; }

// Compression.  In 2-D, two value boxes: the next tile's inputs land (cp.async) in
// one while the passes work on the other, so no load latency sits between two tiles.
template <int NDIM>
__global__ void __launch_bounds__(ND_THREADS, nd_ctas_per_sm<NDIM>()) k_nd_compress(CompressArgs a)
{
    using G = NdGeom<NDIM>;
    __shared__ float vbox[nd_async_stage<NDIM>() ? 2 : 1][vsize<NDIM>(G::BY * G::PX)];
    __shared__ __align__(16) uint16_t cs[hsize<NDIM>(G::TY * G::TX)];
    __shared__ LevelQ lq[ND_MAX_LEVELS];
    extern __shared__ uint32_t hs[];  // histogram bins when 2R <= ND_HIST_SMEM_BINS
    const int tid = threadIdx.x;
    const int bins = 2 * a.radius;
    const bool smem_hist = a.hist && bins <= ND_HIST_SMEM_BINS;
    nd_levels<G::L>(a.hdr, lq);
    if (smem_hist)
        for (int i = tid; i < bins; i += ND_THREADS) hs[i] = 0u;
    const NdCfg cfg = nd_cfg(a.hdr);
    uint32_t central = 0;
    const int tiles = nd_tiles<NDIM>(a.dims);
    constexpr bool ASYNC = nd_async_stage<NDIM>();
    if (ASYNC && (int)blockIdx.x < tiles)
        nd_stage_async<NDIM>(vbox[0], a.x, nd_tile<NDIM>(a.dims, blockIdx.x), a.dims.nx);
    int buf = 0;
    for (int b = blockIdx.x; b < tiles; b += gridDim.x, buf = ASYNC ? buf ^ 1 : 0) {
        if (!ASYNC) {
            const NdTile t = nd_tile<NDIM>(a.dims, b);
            if (t.ey == G::BY - 1 && t.ex == G::BX - 1) nd_stage_full<NDIM>(vbox[0], a.x, t.row0, a.dims.nx, t.x0);
            else nd_stage_clipped<NDIM>(vbox[0], a.x, t.row0, a.dims.nx, t.x0, t.ey, t.ex);
        }
        cp_async_wait_all();
        __syncthreads();  // this tile's box landed (every thread's copies); the other box is free
        const int bn = b + gridDim.x;
        if (ASYNC && bn < tiles) nd_stage_async<NDIM>(vbox[buf ^ 1], a.x, nd_tile<NDIM>(a.dims, bn), a.dims.nx);
        nd_compress_tile<NDIM>(a, cfg, lq, vbox[buf], cs, hs, smem_hist, central, b);
    }
    if (a.hist) {
        const int lane = tid & 31;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) central += __shfl_xor_sync(0xffffffffu, central, off);
        if (lane == 0 && central) atomicAdd(smem_hist ? &hs[a.radius] : &a.hist[a.radius], central);
        if (smem_hist) {
            __syncthreads();
            for (int i = tid; i < bins; i += ND_THREADS)
                if (hs[i]) atomicAdd(&a.hist[i], hs[i]);
        }
    }
}

template <int NDIM>
__device__ __forceinline__ void nd_decompress_tile(const DecompressArgs &a, const NdCfg &cfg, const LevelQ *lq,
                                                   float *v, uint16_t *cb, uint32_t cbias, int b)
{
    using G = NdGeom<NDIM>;
    constexpr int L = G::L;
    const Dims d = a.dims;
    const int tid = threadIdx.x;
    const NdTile t = nd_tile<NDIM>(d, b);

    // the box's codes and anchors (the closing row and column included) were staged by
    // the caller and are visible
    const bool full = t.ey == G::BY - 1 && t.ex == G::BX - 1;

    if (full || NDIM == 2) {
        NdPointCtx c;
        c.cbias = cbias;
        c.cb = cb;
        c.xrec = a.xrec;
        c.row0 = t.row0;
        c.nx = d.nx;
        c.x0 = t.x0;
        if (full) nd_full_tile<NDIM, false>(v, c, lq, cfg);
        else nd2_clipped_tile<false>(v, c, lq, cfg, t.ey, t.ex);
    }
    for (int l = (full || NDIM == 2) ? -1 : L - 1; l >= 0; --l) {
        const int s = 1 << l;
        const float twoe = lq[l].twoe;
        const int spline = cfg.level_kind[l < 2 ? l : 2];
        for (int k = 0; k < 3; ++k) {
            if (cfg.order[k] < 3 - NDIM) continue;
            const NdPass p = nd_pass<NDIM>(t, cfg.order, k, s);
            const Cubic ck = cubic_coeffs(cfg.cubic_kind[p.a]);
            const int npts = p.na * p.no;
            for (int idx = tid; idx < npts; idx += ND_THREADS) {
                int ia, io;
                if (p.a == 2) {
                    ia = idx % p.na;
                    io = idx / p.na;
                } else {
                    io = idx % p.no;
                    ia = idx / p.no;
                }
                const int n = s + 2 * s * ia, m = io * p.so;
                const int i = n * p.sa + m * p.so_mem;
                const float pred = nd_predict<NDIM>(v, i, n, s, p.ea, p.sa, spline, ck);
                const uint32_t code = cb[hix<NDIM>(i)];
                if (code) {
                    v[vix<NDIM>(i)] = pred + code_to_q(code, cbias) * twoe;
                } else {  // outlier: its value was scattered into xrec before this kernel
                    const int by = p.a == 1 ? n : (NDIM == 2 ? m : 0);
                    const int bx = p.a == 2 ? n : m;
                    v[vix<NDIM>(i)] = a.xrec[(t.row0 + by) * d.nx + t.x0 + bx];
                }
            }
            __syncthreads();
        }
    }
    if (t.ox == G::TX && (d.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(a.xrec) & 15u) == 0) {
        // whole-width tiles with 16-byte aligned rows: 4 values per 16-byte store
        constexpr int QPR = G::TX / 4;  // quads per row
        for (int qd = tid; qd < t.oy * QPR; qd += ND_THREADS) {
            const int by = qd / QPR, x4 = 4 * (qd - by * QPR);
            const int j = by * G::PX + x4;
            *reinterpret_cast<float4 *>(a.xrec + (t.row0 + by) * d.nx + t.x0 + x4) =
                make_float4(v[vix<NDIM>(j)], v[vix<NDIM>(j + 1)], v[vix<NDIM>(j + 2)], v[vix<NDIM>(j + 3)]);
        }
    } else {
        for (int by = 0; by < t.oy; ++by) {
            float *dst = a.xrec + (t.row0 + by) * d.nx + t.x0;
            for (int bx = tid; bx < t.ox; bx += ND_THREADS) dst[bx] = v[vix<NDIM>(by * G::PX + bx)];
        }
    }
    __syncthreads();  // the box is reused by the next tile
}

// Decompression.  In 2-D, two code boxes: the next tile's codes land (cp.async) in
// one while the passes read the other, and the next tile's anchors are fetched into
// registers, so no load latency sits between two tiles.  1-D tiles, and fields whose
// rows are not 4-byte aligned, stage the codes with plain loads at each tile's start.
template <int NDIM>
__global__ void __launch_bounds__(ND_THREADS, nd_ctas_per_sm<NDIM>()) k_nd_decompress(DecompressArgs a)
{
    using G = NdGeom<NDIM>;
    __shared__ float v[vsize<NDIM>(G::BY * G::PX)];
    __shared__ __align__(16) uint16_t cbox[nd_async_stage<NDIM>() ? 2 : 1][hsize<NDIM>(G::BY * G::CPX) + 2];
    __shared__ LevelQ lq[ND_MAX_LEVELS];
    nd_levels<G::L>(a.hdr, lq);
    const NdCfg cfg = nd_cfg(a.hdr);
    const uint32_t cbias = kMagicBits - (uint32_t)a.hdr->cfg.radius;
    const int tiles = nd_tiles<NDIM>(a.dims);
    const Dims d = a.dims;
    const bool async =
        nd_async_stage<NDIM>() && (d.nx & 1) == 0 && (reinterpret_cast<uintptr_t>(a.codes) & 3u) == 0;
    float anc = 0.0f;
    int anc_i = 0;
    bool anc_ok = false;
    if (async && (int)blockIdx.x < tiles) {
        const NdTile t = nd_tile<NDIM>(d, blockIdx.x);
        nd_stage_codes_async<NDIM>(cbox[0], a.codes, t, d.nx);
        anc_ok = nd_anchor_fetch<NDIM>(a.anchors, d, t, anc, anc_i);
    }
    int buf = 0;
    for (int b = blockIdx.x; b < tiles; b += gridDim.x, buf = async ? buf ^ 1 : 0) {
        if (!async) {
            const NdTile t = nd_tile<NDIM>(d, b);
            if (t.ey == G::BY - 1 && t.ex == G::BX - 1) nd_stage_full<NDIM>(cbox[buf], a.codes, t.row0, d.nx, t.x0);
            else nd_stage_clipped<NDIM>(cbox[buf], a.codes, t.row0, d.nx, t.x0, t.ey, t.ex);
            anc_ok = nd_anchor_fetch<NDIM>(a.anchors, d, t, anc, anc_i);
        }
        cp_async_wait_all();
        if (anc_ok) v[anc_i] = anc;  // the previous tile ended with a barrier: v is free
        __syncthreads();             // codes landed (every thread's copies), anchors and levels visible
        const int bn = b + gridDim.x;
        anc_ok = false;
        if (async && bn < tiles) {
            const NdTile tn = nd_tile<NDIM>(d, bn);
            nd_stage_codes_async<NDIM>(cbox[buf ^ 1], a.codes, tn, d.nx);
            anc_ok = nd_anchor_fetch<NDIM>(a.anchors, d, tn, anc, anc_i);
        }
        nd_decompress_tile<NDIM>(a, cfg, lq, v, cbox[buf], cbias, b);
    }
}

int nd_tiles_host(int ndim, Dims d)
{
    if (ndim == 2) {
        using G = NdGeom<2>;
        return d.nz * ((d.ny + G::TY - 1) / G::TY) * ((d.nx + G::TX - 1) / G::TX);
    }
    using G = NdGeom<1>;
    return d.nz * d.ny * ((d.nx + G::TX - 1) / G::TX);
}

}  // namespace

cudaError_t launch_nd_compress(int ndim, const CompressArgs &a, cudaStream_t s)
{
    if (ndim != 1 && ndim != 2) return cudaErrorInvalidValue;
    const int tiles = nd_tiles_host(ndim, a.dims);
    if (tiles == 0) return cudaSuccess;
    const size_t hist_smem = (a.hist && 2 * a.radius <= ND_HIST_SMEM_BINS) ? sizeof(uint32_t) * 2 * a.radius : 0;
    const int grid = min(tiles, sm_count() * (ndim == 2 ? nd_ctas_per_sm<2>() : nd_ctas_per_sm<1>()));
    if (ndim == 2)
        k_nd_compress<2><<<grid, ND_THREADS, hist_smem, s>>>(a);
    else
        k_nd_compress<1><<<grid, ND_THREADS, hist_smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nd_decompress(int ndim, const DecompressArgs &a, cudaStream_t s)
{
    if (ndim != 1 && ndim != 2) return cudaErrorInvalidValue;
    const int tiles = nd_tiles_host(ndim, a.dims);
    if (tiles == 0) return cudaSuccess;
    const int grid = min(tiles, sm_count() * (ndim == 2 ? nd_ctas_per_sm<2>() : nd_ctas_per_sm<1>()));
    if (ndim == 2)
        k_nd_decompress<2><<<grid, ND_THREADS, 0, s>>>(a);
    else
        k_nd_decompress<1><<<grid, ND_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gi
