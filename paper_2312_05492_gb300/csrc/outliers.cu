// Outlier stream compaction (Sec. V-A: outliers are gathered and stored
// losslessly), the outlier scatter of decompression, and the standalone
// quant-code histogram (Fig. 1 "histogram", Sec. V-A).
//
// Compaction is ordered: the compression kernel writes one bitmap word per
// 32 x-positions of every row and adds the popcount of each non-zero word to
// the counter of its 2048-word block.  A one-CTA scan turns the block counts
// into offsets, then one CTA per non-empty block expands its words into
// (index, value) pairs.  Words are in ascending linear-index order, so the
// outlier list comes out sorted by index with no sort and no atomics.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace gi {
namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int WRITE_THREADS = 256;
constexpr int WORDS_PER_THREAD = BITMAP_BLOCK_WORDS / WRITE_THREADS;  // 8
static_assert(WORDS_PER_THREAD * WRITE_THREADS == BITMAP_BLOCK_WORDS, "block geometry");

// Exclusive scan of the block counts in place; total -> header.  With a
// histogram whose central bin R the tile kernel left out (it is the most
// frequent code by far), the bin is filled in here: N minus every other bin.
__device__ void outlier_scan_block(uint32_t *blockcnt, int nblk, interp_header *hdr, unsigned long long capacity,
                                   uint32_t *hist, int radius, unsigned long long n)
{
    __shared__ unsigned long long warp_sum[SCAN_THREADS / 32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += SCAN_THREADS) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < nblk ? blockcnt[i] : 0u;
        unsigned long long incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            warp_sum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? warp_sum[warp - 1] : 0ull) + incl - v;
        // offsets of blocks fit in 32 bits because N < 2^32
        if (i < nblk) blockcnt[i] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hdr->n_outliers = carry;
        if (carry > capacity) hdr->status |= INTERP_STATUS_CAPACITY;
    }
    if (hist) {
        unsigned long long others = 0;
        for (int c = threadIdx.x; c < 2 * radius; c += SCAN_THREADS)
            if (c != radius) others += hist[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) others += __shfl_xor_sync(0xffffffffu, others, off);
        __syncthreads();
        if (lane == 0) warp_sum[warp] = others;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) t += warp_sum[w];
            hist[radius] = (uint32_t)(n - t);
        }
    }
}

__device__ void outlier_write_block(const uint32_t *__restrict__ bitmap, const uint32_t *__restrict__ offsets,
                                    long long words, int words_per_row, int nx, int ny, int nz,
                                    const float *__restrict__ x, uint32_t *out_idx, float *out_val,
                                    unsigned long long capacity, const interp_header *hdr, int nblk, bool row_major,
                                    int b)
{
    const unsigned long long total = hdr->n_outliers;
    const unsigned long long start = offsets[b];
    const unsigned long long end = (b + 1 < nblk) ? offsets[b + 1] : total;
    if (end == start || start >= capacity) return;  // empty block, or beyond the caller's capacity

    const long long w0 = (long long)b * BITMAP_BLOCK_WORDS + (long long)threadIdx.x * WORDS_PER_THREAD;
    uint32_t wv[WORDS_PER_THREAD];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < WORDS_PER_THREAD; ++k) {
        const long long w = w0 + k;
        wv[k] = (w < words) ? bitmap[row_major ? (size_t)w : tiled_word(w, words_per_row, ny, nz)] : 0u;
        cnt += __popc(wv[k]);
    }
    // block exclusive scan of per-thread counts
    __shared__ int warp_sum[WRITE_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = incl - cnt;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];

    unsigned long long pos = start + (unsigned long long)before;
#pragma unroll
    for (int k = 0; k < WORDS_PER_THREAD; ++k) {
        uint32_t m = wv[k];
        if (!m) continue;
        const long long wi = w0 + k;
        const long long row = wi / words_per_row;
        const long long xb = (wi % words_per_row) * 32;
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            if (pos < capacity) {
                const unsigned long long idx = (unsigned long long)row * nx + xb + bit;
                out_idx[pos] = (uint32_t)idx;
                out_val[pos] = x[idx];
            }
            ++pos;
        }
    }
}

// Ordered compaction of the outliers of n fields in two launches: one scan block
// per field, then every field's non-empty bitmap blocks.
struct CompactField {
    const uint32_t *bitmap;
    uint32_t *blockcnt;
    long long words;
    int words_per_row, nx, ny, nz;
    const float *x;
    uint32_t *out_idx;
    float *out_val;
    unsigned long long capacity;
    interp_header *hdr;
    int nblk;
    bool row_major;
    uint32_t *hist;  // fills bin R when not null
    int radius;
    unsigned long long n;
    int b0;          // first write block of the field
};

struct CompactBatch {
    CompactField f[kMaxBatch];
    int n;
};

__global__ void __launch_bounds__(SCAN_THREADS) k_outlier_scan(const __grid_constant__ CompactBatch B)
{
    const CompactField &F = B.f[blockIdx.x];
    outlier_scan_block(F.blockcnt, F.nblk, F.hdr, F.capacity, F.hist, F.radius, F.n);
}

__global__ void __launch_bounds__(WRITE_THREADS) k_outlier_write(const __grid_constant__ CompactBatch B)
{
    int fi = 0;
    while (fi + 1 < B.n && B.f[fi + 1].b0 <= (int)blockIdx.x) ++fi;
    const CompactField &F = B.f[fi];
    outlier_write_block(F.bitmap, F.blockcnt, F.words, F.words_per_row, F.nx, F.ny, F.nz, F.x, F.out_idx,
                        F.out_val, F.capacity, F.hdr, F.nblk, F.row_major, (int)blockIdx.x - F.b0);
}

// Outlier values of n fields into their reconstructions: `blocks` blocks per field.
struct ScatterField {
    const interp_header *hdr;
    const uint32_t *idx;
    const float *val;
    unsigned long long capacity;
    float *xrec;
};

struct ScatterBatch {
    ScatterField f[kMaxBatch];
    int n, blocks;
};

__global__ void k_outlier_scatter(const __grid_constant__ ScatterBatch B)
{
    const ScatterField &F = B.f[blockIdx.x / B.blocks];
    const unsigned long long b = blockIdx.x % B.blocks;
    unsigned long long n = F.hdr->n_outliers;
    if (n > F.capacity) n = F.capacity;
    for (unsigned long long i = b * blockDim.x + threadIdx.x; i < n; i += (unsigned long long)B.blocks * blockDim.x)
        F.xrec[F.idx[i]] = F.val[i];
}

// Standalone histogram: per-CTA shared bins (register count for the central
// code R, which dominates for accurate predictions, Sec. V-A), flushed once.
constexpr int HIST_THREADS = 512;
constexpr int HIST_SMEM_MAX_BINS = 16384;

__global__ void __launch_bounds__(HIST_THREADS) k_histogram(const uint16_t *__restrict__ codes,
                                                            unsigned long long n, int radius, int vec,
                                                            uint32_t *hist)
{
    extern __shared__ uint32_t hs[];
    const int bins = 2 * radius;
    const bool smem = bins <= HIST_SMEM_MAX_BINS;
    if (smem)
        for (int i = threadIdx.x; i < bins; i += HIST_THREADS) hs[i] = 0u;
    __syncthreads();
    uint32_t central = 0;
    auto count = [&](uint32_t c) {
        if (c == (uint32_t)radius) {
            ++central;
        } else if (c < (uint32_t)bins) {
            if (smem) atomicAdd(&hs[c], 1u);
            else atomicAdd(&hist[c], 1u);
        }
    };
    const unsigned long long tid = (unsigned long long)blockIdx.x * HIST_THREADS + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * HIST_THREADS;
    unsigned long long done = 0;
    if (vec) {
        const uint4 *c8 = reinterpret_cast<const uint4 *>(codes);
        const unsigned long long n8 = n / 8;
        for (unsigned long long i = tid; i < n8; i += nth) {
            const uint4 v = __ldcs(c8 + i);
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                count(w4[k] & 0xffffu);
                count(w4[k] >> 16);
            }
        }
        done = n8 * 8;
    }
    for (unsigned long long i = done + tid; i < n; i += nth) count(codes[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) central += __shfl_xor_sync(0xffffffffu, central, off);
    if ((threadIdx.x & 31) == 0 && central) {
        if (smem) atomicAdd(&hs[radius], central);
        else atomicAdd(&hist[radius], central);
    }
    if (smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += HIST_THREADS) {
            const uint32_t h = hs[i];
            if (h) atomicAdd(&hist[i], h);
        }
    }
}

}  // namespace

cudaError_t launch_outlier_compaction(const CompactItem *items, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    CompactBatch B;
    std::memset(&B, 0, sizeof(B));
    int blocks = 0;
    for (int i = 0; i < n; ++i) {
        const CompactItem &it = items[i];
        CompactField &F = B.f[i];
        F.bitmap = it.bitmap;
        F.blockcnt = it.blockcnt;
        F.words = (long long)it.words;
        F.words_per_row = (it.d.nx + 31) / 32;
        F.nx = it.d.nx;
        F.ny = it.d.ny;
        F.nz = it.d.nz;
        F.x = it.x;
        F.out_idx = it.out_idx;
        F.out_val = it.out_val;
        F.capacity = (unsigned long long)it.capacity;
        F.hdr = it.hdr;
        F.nblk = (int)((it.words + BITMAP_BLOCK_WORDS - 1) / BITMAP_BLOCK_WORDS);
        F.row_major = it.row_major;
        F.hist = it.central_hist;
        F.radius = it.radius;
        F.n = (unsigned long long)it.d.nz * it.d.ny * it.d.nx;
        F.b0 = blocks;
        blocks += F.nblk;
    }
    B.n = n;
    k_outlier_scan<<<n, SCAN_THREADS, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_outlier_write<<<blocks, WRITE_THREADS, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_outlier_scatter(const ScatterItem *items, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    ScatterBatch B;
    std::memset(&B, 0, sizeof(B));
    for (int i = 0; i < n; ++i) B.f[i] = ScatterField{items[i].hdr, items[i].idx, items[i].val,
                                                      (unsigned long long)items[i].capacity, items[i].xrec};
    B.n = n;
    B.blocks = std::max(1, 2 * sm_count() / n);
    k_outlier_scatter<<<B.blocks * n, 256, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const uint16_t *codes, uint64_t n, int radius, uint32_t *hist, cudaStream_t s)
{
    const int bins = 2 * radius;
    const size_t smem = bins <= HIST_SMEM_MAX_BINS ? sizeof(uint32_t) * (size_t)bins : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int vec = (reinterpret_cast<uintptr_t>(codes) % 16) == 0;
    unsigned long long blocks = (n + 8ull * HIST_THREADS * 8 - 1) / (8ull * HIST_THREADS * 8);
    const unsigned long long cap = 4ull * sm_count();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_histogram<<<(unsigned)blocks, HIST_THREADS, smem, s>>>(codes, (unsigned long long)n, radius, vec, hist);
    return cudaGetLastError();
}

}  // namespace gi
