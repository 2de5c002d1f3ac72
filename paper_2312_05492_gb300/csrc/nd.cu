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
// One CTA per tile: 2-D tiles own 16 rows x 128 columns of one slice, 1-D tiles
// 2048 points of one row; the CTA stages the tile with its closing row and column
// (the anchors and points its chunks borrow from the next tile) in shared memory,
// runs every pass on it, and writes only what it owns.  Passes inside a tile are
// separated by barriers; tiles are independent.
//
// Outputs match the 3-D path's formats: codes (q + R, 0 for outliers, R at
// anchors), anchors [nz'][ny'][nx'], the fused histogram, and the outlier bitmap
// (one word per 32 x-positions of a row, tile-major addresses) with per-block
// popcounts for the ordered compaction.
#include "common.cuh"

namespace gi {
namespace {

constexpr int ND_THREADS = 256;
constexpr int ND_MAX_LEVELS = 9;
constexpr int ND_HIST_SMEM_BINS = 8192;

template <int NDIM>
struct NdGeom;
template <>
struct NdGeom<2> {
    static constexpr int A = 16, L = 4;
    static constexpr int TY = 16, TX = 128;    // owned rows x columns
    static constexpr int BY = 17, BX = 129;    // staged box
    static constexpr int PX = 129;             // row pitch (odd: column walks hit distinct banks)
};
template <>
struct NdGeom<1> {
    static constexpr int A = 512, L = 9;
    static constexpr int TY = 1, TX = 2048;
    static constexpr int BY = 1, BX = 2049;
    static constexpr int PX = 2049;
};

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
    double apow = 1.0;
    for (int l = 0; l < L; ++l) {
        const float e = (float)(h->eb_abs / apow);
        lq[l] = LevelQ{e, 2.0f * e, (float)(1.0 / (2.0 * (double)e))};
        apow *= h->alpha;
    }
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
template <int A>
__device__ __forceinline__ float nd_predict(const float *v, int i, int n, int s, int ea, int sa, int spline,
                                           const Cubic &ck)
{
    const int lo = (n / A) * A;
    const int hi = min(lo + A, ea);
    const float m1 = v[i - s * sa];
    if (n + s > hi) return m1;
    const float p1 = v[i + s * sa];
    if (!spline) return sp_linear(m1, p1);
    const bool has_m3 = n - 3 * s >= lo, has_p3 = n + 3 * s <= hi;
    if (has_m3 && has_p3) return sp_cubic(ck, v[i - 3 * s * sa], m1, p1, v[i + 3 * s * sa]);
    if (has_m3) return sp_quad_left(v[i - 3 * s * sa], m1, p1);
    if (has_p3) return sp_quad_right(m1, p1, v[i + 3 * s * sa]);
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

template <int NDIM>
__global__ void __launch_bounds__(ND_THREADS) k_nd_compress(CompressArgs a)
{
    using G = NdGeom<NDIM>;
    constexpr int L = G::L;
    __shared__ float v[G::BY * G::PX];
    __shared__ uint16_t cs[G::TY * G::TX];
    __shared__ LevelQ lq[ND_MAX_LEVELS];
    extern __shared__ uint32_t hs[];  // histogram bins when 2R <= ND_HIST_SMEM_BINS
    const Dims d = a.dims;
    const interp_header *h = a.hdr;
    const int tid = threadIdx.x;
    const int bins = 2 * a.radius;
    const bool smem_hist = a.hist && bins <= ND_HIST_SMEM_BINS;
    if (tid == 0) nd_levels<L>(h, lq);
    if (smem_hist)
        for (int i = tid; i < bins; i += ND_THREADS) hs[i] = 0u;
    const NdCfg cfg = nd_cfg(h);
    const uint32_t cbias = kMagicBits - (uint32_t)a.radius;
    const float Rf = (float)a.radius;
    const NdTile t = nd_tile<NDIM>(d, blockIdx.x);

    // stage the box
    for (int by = 0; by <= t.ey; ++by) {
        const float *src = a.x + (t.row0 + by) * d.nx + t.x0;
        for (int bx = tid; bx <= t.ex; bx += ND_THREADS) v[by * G::PX + bx] = __ldg(src + bx);
    }
    // owned anchors: code R, value kept
    for (int i = tid; i < G::TY * G::TX; i += ND_THREADS) cs[i] = (uint16_t)a.radius;
    __syncthreads();

    for (int l = L - 1; l >= 0; --l) {
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
                const float pred = nd_predict<G::A>(v, i, n, s, p.ea, p.sa, spline, ck);
                float xr;
                const uint32_t code = quantize(v[i], pred, q, cbias, Rf, xr);
                v[i] = xr;
                const int by = p.a == 1 ? n : (NDIM == 2 ? m : 0);
                const int bx = p.a == 2 ? n : m;
                if (by < G::TY && bx < G::TX) cs[by * G::TX + bx] = (uint16_t)code;
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
                a.anchors[arow * ax + (t.x0 + bx) / G::A] = v[bx];
    }

    // codes, outlier bitmap words and the histogram of the owned points, one
    // 32-column strip of a row per warp step
    const int lane = tid & 31, warp = tid >> 5;
    const int wpr = (d.nx + 31) / 32;
    const int strips = (t.ox + 31) / 32;
    uint32_t central = 0;
    for (int u = warp; u < t.oy * strips; u += ND_THREADS / 32) {
        const int by = u / strips, bx = (u - by * strips) * 32 + lane;
        const bool in = bx < t.ox;
        const uint32_t code = in ? cs[by * G::TX + bx] : 1u;
        const long long row = t.row0 + by;
        if (in) a.codes[row * d.nx + t.x0 + bx] = (uint16_t)code;
        const uint32_t word = __ballot_sync(0xffffffffu, code == 0u);
        if (lane == 0) {
            const long long gw = row * wpr + (t.x0 >> 5) + (bx >> 5);
            a.bitmap[tiled_word(gw, wpr, d.ny, d.nz)] = word;
            if (word) atomicAdd(a.blockcnt + gw / BITMAP_BLOCK_WORDS, (uint32_t)__popc(word));
        }
        if (a.hist && in) {
            if (code == (uint32_t)a.radius) ++central;
            else if (code < (uint32_t)bins) atomicAdd(smem_hist ? &hs[code] : &a.hist[code], 1u);
        }
    }
    if (a.hist) {
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
__global__ void __launch_bounds__(ND_THREADS) k_nd_decompress(DecompressArgs a)
{
    using G = NdGeom<NDIM>;
    constexpr int L = G::L;
    __shared__ float v[G::BY * G::PX];
    __shared__ uint16_t cb[G::BY * G::PX];
    __shared__ LevelQ lq[ND_MAX_LEVELS];
    const Dims d = a.dims;
    const interp_header *h = a.hdr;
    const int tid = threadIdx.x;
    if (tid == 0) nd_levels<L>(h, lq);
    const NdCfg cfg = nd_cfg(h);
    const uint32_t cbias = kMagicBits - (uint32_t)h->cfg.radius;
    const NdTile t = nd_tile<NDIM>(d, blockIdx.x);

    // stage the box's codes and anchors (the closing row and column included)
    const int ax = (d.nx - 1) / G::A + 1;
    for (int by = 0; by <= t.ey; ++by) {
        const uint16_t *src = a.codes + (t.row0 + by) * d.nx + t.x0;
        for (int bx = tid; bx <= t.ex; bx += ND_THREADS) cb[by * G::PX + bx] = __ldg(src + bx);
        const bool anchor_row = NDIM == 1 || (t.y0 + by) % G::A == 0;
        if (anchor_row) {
            const long long arow =
                NDIM == 2 ? (long long)t.z * ((d.ny - 1) / G::A + 1) + (t.y0 + by) / G::A : t.row0;
            for (int bx = tid * G::A; bx <= t.ex; bx += ND_THREADS * G::A)
                v[by * G::PX + bx] = __ldg(a.anchors + arow * ax + (t.x0 + bx) / G::A);
        }
    }
    __syncthreads();

    for (int l = L - 1; l >= 0; --l) {
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
                const float pred = nd_predict<G::A>(v, i, n, s, p.ea, p.sa, spline, ck);
                const uint32_t code = cb[i];
                if (code) {
                    v[i] = pred + code_to_q(code, cbias) * twoe;
                } else {  // outlier: its value was scattered into xrec before this kernel
                    const int by = p.a == 1 ? n : (NDIM == 2 ? m : 0);
                    const int bx = p.a == 2 ? n : m;
                    v[i] = a.xrec[(t.row0 + by) * d.nx + t.x0 + bx];
                }
            }
            __syncthreads();
        }
    }
    for (int by = 0; by < t.oy; ++by) {
        float *dst = a.xrec + (t.row0 + by) * d.nx + t.x0;
        for (int bx = tid; bx < t.ox; bx += ND_THREADS) dst[bx] = v[by * G::PX + bx];
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
    if (ndim == 2)
        k_nd_compress<2><<<tiles, ND_THREADS, hist_smem, s>>>(a);
    else
        k_nd_compress<1><<<tiles, ND_THREADS, hist_smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nd_decompress(int ndim, const DecompressArgs &a, cudaStream_t s)
{
    if (ndim != 1 && ndim != 2) return cudaErrorInvalidValue;
    const int tiles = nd_tiles_host(ndim, a.dims);
    if (tiles == 0) return cudaSuccess;
    if (ndim == 2)
        k_nd_decompress<2><<<tiles, ND_THREADS, 0, s>>>(a);
    else
        k_nd_decompress<1><<<tiles, ND_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gi
