// Shared device-side definitions of the G-Interp CUDA library (sm_103a).
//
// Every kernel is compiled with --fmad=false: each float operation below is
// rounded on its own, in the order written, so the quant-codes and the
// reconstruction are reproducible bit for bit.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "ginterp.h"

namespace gi {

// ----------------------------------------------------------- tile geometry
// A CTA works on a tile of TZ x TY x TX chunks of 8^3 points (Sec. IV-A),
// staged in shared memory together with the closing faces at the far end of
// each axis (the "borrowed" anchors and face points of the neighbouring
// chunks, Sec. IV-C), i.e. a (8TZ+1) x (8TY+1) x (8TX+1) box.
// A CTA marches along z through a column of 2 x 4 chunks of 8^3 points
// (16 y x 32 x owned points), one slab of 8 planes at a time.
#ifndef GI_TILE_THREADS
#define GI_TILE_THREADS 192
#endif
#ifndef GI_TILE_ROWS
#define GI_TILE_ROWS 16
#endif
constexpr int OY = GI_TILE_ROWS, OX = 32;  // owned extent of a column
static_assert(OY % 8 == 0, "columns hold whole chunks");
constexpr int TILE_THREADS = GI_TILE_THREADS;
static_assert(OX == 32, "one outlier-bitmap word covers the 32 x-positions of an owned row");

// outlier bitmap: one 32-bit word per 32 x-positions of every (z, y) row
constexpr int BITMAP_BLOCK_WORDS = 2048;  // words per compaction block

// histogram bins kept in shared memory by the fused histogram
constexpr int HIST_SMEM_BINS = 1024;

// fields per batched call (one persistent tile launch covers all of them)
constexpr int kMaxBatch = 16;

// ------------------------------------------------------------- parameters
struct Dims {
    int nz, ny, nx;
};

struct TileGrid {
    int tz, ty, tx;  // tiles per axis
};

// ---------------------------------------------------------------- splines
// p for the neighbour sets of Sec. IV-B.1; m3, m1, p1, p3 = x_{n-3s}, x_{n-s},
// x_{n+s}, x_{n+3s}.
__device__ __forceinline__ float sp_linear(float m1, float p1) { return (m1 + p1) * 0.5f; }
__device__ __forceinline__ float sp_quad_left(float m3, float m1, float p1)
{
    return ((6.0f * m1 - m3) + 3.0f * p1) * 0.125f;
}
__device__ __forceinline__ float sp_quad_right(float m1, float p1, float p3)
{
    return ((3.0f * m1 + 6.0f * p1) - p3) * 0.125f;
}
// Cubic splines: the integer-weighted sum over the printed denominator, i.e.
// not-a-knot (9(m1+p1) - (m3+p3)) / 16, a multiply by 0.0625 (exact: a power of
// two), and natural (23(m1+p1) - 3(m3+p3)) / 40, an IEEE division.
__device__ __forceinline__ float sp_cubic_nak(float m3, float m1, float p1, float p3)
{
    return (9.0f * (m1 + p1) - (m3 + p3)) * 0.0625f;
}
// n / 40 rounded to nearest even, exactly as an IEEE division would give it.
// Normal range: q = n * RN(1/40) is within one ulp of n / 40, the residual
// n - 40 q is exact as one fused multiply-add, and q + residual * RN(1/40) is
// the correctly rounded quotient (Markstein's correction step, P. Markstein,
// IBM J. Res. Dev. 34(1), 1990).  Tiny numerators are scaled by 2^64 first
// (the scaled quotient is normal and scaling back is exact while n / 40 stays
// normal); numerators whose quotient is subnormal are divided in integers, in
// units of 2^-149, with the remainder deciding the rounding.  Checked against
// CUDA's IEEE division on every float input.
__device__ __forceinline__ float div40_markstein(float n)
{
    const float y = 0.025f;  // RN(1/40)
    const float q = __fmul_rn(n, y);
    const float r = __fmaf_rn(-q, 40.0f, n);
    return __fmaf_rn(r, y, q);
}
__device__ __forceinline__ float div40_tiny(float n)
{
    const float a = fabsf(n);
    if (!(a <= 3.402823466e38f)) return __fmul_rn(n, 0.025f);  // inf / 40 = inf; NaN stays NaN
    if (a >= 4.70197740e-37f)  // 40 * 2^-126: the quotient is normal
        return __fmul_rn(div40_markstein(__fmul_rn(n, 18446744073709551616.0f)), 5.42101086e-20f);  // 2^64, 2^-64
    // quotient below 2^-126: |n| = M * 2^-149 with M < 2^29, the result is round(M / 40) * 2^-149
    const uint32_t M = (uint32_t)__fmul_rn(__fmul_rn(a, 1.26765060e30f), 5.62949953e14f);  // * 2^100 * 2^49: exact
    uint32_t qi = M / 40u;
    const uint32_t rem = M - 40u * qi;
    if (rem > 20u || (rem == 20u && (qi & 1u))) ++qi;
    return __uint_as_float((__float_as_uint(n) & 0x80000000u) | qi);
}
__device__ __forceinline__ float div40_rn(float n)
{
    const float a = fabsf(n);
    return (a >= 8.07793567e-28f && a <= 3.402823466e38f) ? div40_markstein(n) : div40_tiny(n);  // 2^-90 .. max
}
__device__ __forceinline__ float sp_cubic_nat(float m3, float m1, float p1, float p3)
{
    return div40_rn(23.0f * (m1 + p1) - 3.0f * (m3 + p3));
}
// the cubic kind chosen at run time (0 = not-a-knot, 1 = natural)
struct Cubic {
    int natural;
};
__device__ __forceinline__ Cubic cubic_coeffs(int natural) { return Cubic{natural ? 1 : 0}; }
__device__ __forceinline__ float sp_cubic(const Cubic &k, float m3, float m1, float p1, float p3)
{
    return k.natural ? sp_cubic_nat(m3, m1, p1, p3) : sp_cubic_nak(m3, m1, p1, p3);
}

// Level-wise quantization constants, read once per CTA from the header.
struct LevelQ {
    float e, twoe, inv2e;
};

// Rounding by the float adder: for |v| < 2^22, v + 1.5*2^23 lies in
// (2^23, 2^24), where floats are spaced by 1, so the sum rounds v to an
// integer with ties to even (1.5*2^23 is even): (v + kMagic) - kMagic is
// exactly rintf(v), and the bits of v + kMagic are kMagicBits + rintf(v).
// For |v| >= 2^22 the result has magnitude >= 2^22 > R, so the point is an
// outlier exactly when it is one with rintf; NaN and Inf propagate.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;

// Quantize x against prediction p (Sec. III-A): q = rint((x - p) / 2e);
// kept iff |q| < R and the reconstruction p + q*2e is within e of x.
// Returns the code (q + R, or 0 for an outlier) and writes x' to xr.
// cbias = kMagicBits - R.
__device__ __forceinline__ uint32_t quantize(float x, float p, const LevelQ &L, uint32_t cbias, float Rf, float &xr)
{
    const float d = x - p;
    const float v = d * L.inv2e;
    const float y = v + kMagic;
    const float q = y - kMagic;
    bool ok = fabsf(q) < Rf;
    const float r = p + q * L.twoe;
    ok = ok && (fabsf(x - r) <= L.e);
    xr = ok ? r : x;
    return ok ? __float_as_uint(y) - cbias : 0u;
}

// (code - R) as a float, exactly (|code - R| < 2^22): the float whose bits are
// kMagicBits + (code - R) is kMagic + (code - R).
__device__ __forceinline__ float code_to_q(uint32_t code, uint32_t cbias)
{
    return __uint_as_float(code + cbias) - kMagic;
}

}  // namespace gi

// ------------------------------------------------------------- launchers
// (C++ linkage, internal to the library; the C ABI lives in abi.cu)
namespace gi {

struct CompressArgs {
    const float *x;
    Dims dims;
    float *anchors;
    uint16_t *codes;
    uint32_t *bitmap;
    uint32_t *blockcnt;
    uint32_t *hist;  // may be null
    int radius;
    interp_header *hdr;
    bool vec_codes;  // codes 16-byte aligned and nx % 8 == 0: 8-code vector stores
    bool xdom32;     // x-extended neighbour domain requested (cfg.domain_x == 32)
    int code_store;  // codes per store on rows of 8 codes starting at x = 8k: 8, 4 or 2
                     // (by the alignment of codes and nx), else 1
};

struct DecompressArgs {
    Dims dims;
    const float *anchors;
    const uint16_t *codes;
    float *xrec;
    const interp_header *hdr;
    bool vec_xrec;  // xrec 16-byte aligned and nx % 4 == 0: 4-value vector stores
    const uint32_t *out_idx = nullptr;  // the outlier list (ascending indices), may be null
    uint64_t out_capacity = 0;          // its length in entries
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Bitmap word gw (ascending index order: row = gw / words_per_row of the (z, y)
// rows, 32 x-positions each) lives at a tile-major address: rows are grouped by
// OY along y, and a group's words of one 32-column strip are contiguous per z.
__device__ __forceinline__ size_t tiled_word(long long gw, int words_per_row, int ny, int nz)
{
    const long long row = gw / words_per_row;
    const int cx = (int)(gw - row * words_per_row);
    const int gz = (int)(row / ny), gy = (int)(row - (long long)gz * ny);
    const size_t col = (size_t)(gy / OY) * words_per_row + cx;
    return (col * nz + gz) * OY + (gy % OY);
}

cudaError_t launch_header_init(interp_header *hdr, Dims d, double eb, interp_config cfg, double alpha,
                               cudaStream_t s);
// compression set-up of n fields (1 <= n <= kMaxBatch) in two launches: zero the
// control words, block counters and histogram of every field, then profile +
// decision (autotune) and value range + bounds (relative) or bounds (absolute)
struct PrologueItem {
    const float *x;
    Dims d;
    double eb;
    interp_config cfg;
    double alpha;
    interp_header *hdr;
    uint32_t *counter;  // the workspace's control words (the range counter is the first)
    int ctrl_words;
    void *partials;
    uint32_t *blockcnt;
    int nblk;
    uint32_t *hist;     // may be null
};
cudaError_t launch_prologue(const PrologueItem *items, int n, cudaStream_t s);
cudaError_t launch_profile(const float *x, Dims d, interp_header *hdr, int apply_decision, cudaStream_t s,
                           int ndim = 3);
cudaError_t launch_range(const float *x, Dims d, double eb, interp_config cfg, double alpha, interp_header *hdr,
                         void *partials, unsigned int *counter, int nblocks, cudaStream_t s,
                         float *out_range = nullptr);  // hdr == nullptr: write {vmin, vmax} to out_range
// one persistent launch over the tiles of n fields (1 <= n <= kMaxBatch)
// schedule of a persistent tile launch: slabs per work item and CTAs per SM (0 = automatic)
struct TileSchedule {
    int run;
    int ctas_per_sm;
};
cudaError_t launch_compress_tiles(const CompressArgs *args, int n, cudaStream_t s,
                                  const TileSchedule *sched = nullptr);
cudaError_t launch_decompress_tiles(const DecompressArgs *args, int n, cudaStream_t s,
                                    const TileSchedule *sched = nullptr);
size_t bitmap_words_tiled(Dims d);
// 1-D (512-point chunks) and 2-D (16^2 chunks) variants (nd.cu); ndim 1 or 2
cudaError_t launch_nd_compress(int ndim, const CompressArgs &a, cudaStream_t s);
cudaError_t launch_nd_decompress(int ndim, const DecompressArgs &a, cudaStream_t s);
// ordered outlier compaction of n fields (one scan launch, one write launch)
struct CompactItem {
    const uint32_t *bitmap;
    uint32_t *blockcnt;
    int64_t words;
    Dims d;
    const float *x;
    uint32_t *out_idx;
    float *out_val;
    uint64_t capacity;
    interp_header *hdr;
    bool row_major;          // bitmap in row-major order (1-D / 2-D kernels), else tile-major
    uint32_t *central_hist;  // not null: fill bin R as N minus the other bins
    int radius;
};
cudaError_t launch_outlier_compaction(const CompactItem *items, int n, cudaStream_t s);
// outlier values of n fields into their reconstructions (one launch)
struct ScatterItem {
    const interp_header *hdr;
    const uint32_t *idx;
    const float *val;
    uint64_t capacity;
    float *xrec;
};
cudaError_t launch_outlier_scatter(const ScatterItem *items, int n, cudaStream_t s);
cudaError_t launch_histogram(const uint16_t *codes, uint64_t n, int radius, uint32_t *hist, cudaStream_t s);

cudaError_t launch_quality(const uint32_t *hist, int radius, const float *x, const float *xr, uint64_t n,
                           interp_quality *out, void *ws, cudaStream_t s);
size_t quality_workspace_bytes();

// canonical Huffman coding of the codes (huffman.cu)
bool huffman_codebook(const uint32_t *hist, int nsym, int max_len, uint8_t *lengths, uint32_t *codewords);
unsigned long long huffman_chunks(unsigned long long n);
unsigned long long huffman_capacity_words(unsigned long long n, int max_len);
size_t huffman_decode_workspace(int nsym);
int huffman_max_len();
size_t huffman_encode_workspace(unsigned long long n);  // per-CTA word counts of the encoder
cudaError_t launch_huffman_encode(const uint16_t *codes, unsigned long long n, const uint8_t *lengths,
                                  const uint32_t *codewords, int nsym, uint32_t *offsets, uint32_t *words,
                                  unsigned long long capacity_words, uint32_t *block_words, unsigned int *bad,
                                  cudaStream_t s);
cudaError_t launch_huffman_decode(const uint32_t *words, const uint32_t *offsets, unsigned long long n,
                                  const uint8_t *lengths, const uint32_t *codewords, int nsym, uint16_t *codes,
                                  void *ws, unsigned int *bad, cudaStream_t s);

int range_blocks();
int sm_count();

}  // namespace gi
