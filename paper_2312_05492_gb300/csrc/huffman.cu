// Canonical Huffman coding of the quant-codes: the lossless stage that follows
// the histogram (Sec. V-A: the codebook is built on the host from the histogram,
// the codes are encoded and decoded on the GPU).
//
// Stream format: the codes are cut into chunks of 1024 consecutive codes; a
// chunk's codewords are concatenated most-significant bit first into 32-bit
// words (its first bit is bit 31 of its first word) and padded with zero bits
// to a whole word; offsets[k] is chunk k's first word, offsets[nchunks] the
// total.  Chunks start on word boundaries, so they decode independently.
//
// Encoding: one warp per chunk, each lane 32 consecutive codes, ENC_WARPS chunks
// per CTA.  A first pass sums the code lengths of each CTA's chunks (in words), a
// one-CTA scan turns those sums into word offsets, and a second pass recomputes
// its chunks' sizes, places them after the CTA's offset, and has every lane put
// its codewords at its bit offset (a warp scan) in the warp's shared-memory copy
// of the chunk, which is then written out with coalesced stores.
// Decoding: one thread per chunk, reading its words in order: the next 10 bits
// index a lookup table holding every whole codeword they contain (up to three
// symbols and the bits they take); longer codewords take the canonical rule (per
// length, the first codeword and the first symbol index).  Decoded codes are
// staged per warp and stored coalesced.
#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include "common.cuh"

namespace gi {
namespace {


constexpr int HCHUNK = 1024;          // codes per chunk
constexpr int HLANE = HCHUNK / 32;    // codes per lane
constexpr int ENC_WARPS = 8;
constexpr int ENC_THREADS = 32 * ENC_WARPS;
constexpr int MAX_LEN = 24;           // longest codeword the library builds
constexpr int LUT_BITS = 10;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int TAB_THREADS = 1024;
constexpr int DEC_ROUND = 32;  // codes a decoding thread stages before its warp stores them
constexpr int SYM_SMEM = 8192; // canonical symbol list kept in shared memory up to this many symbols
constexpr int DEC_THREADS = 128;

// Device decode tables, built per call from the code lengths.
struct DecodeTables {
    uint32_t first[MAX_LEN + 2];      // first codeword of each length (canonical)
    uint32_t count[MAX_LEN + 2];      // codewords of each length
    uint32_t base[MAX_LEN + 2];       // index in `symbols` of each length's first symbol
    // The whole codewords (up to 3) that the next LUT_BITS bits hold: bits 0-15, 16-31,
    // 32-47 the symbols, 48-51 / 52-55 / 56-59 the bits consumed after 1 / 2 / 3 of
    // them, 60-61 their number (0: the first codeword is longer than LUT_BITS).
    unsigned long long lut[1 << LUT_BITS];
    int max_len;
};
// followed by uint16_t symbols[2R] in canonical order

// A lane's 32 consecutive codes (64 bytes) as four 16-byte loads when the chunk is
// whole and the codes array is 16-byte aligned; c[j] is code j of the lane.
__device__ __forceinline__ int lane_codes(const uint16_t *__restrict__ codes, unsigned long long n,
                                          unsigned long long i0, bool vec, uint32_t w[16])
{
    if (vec && i0 + HLANE <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(codes + i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 v = __ldg(p + k);
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
        return HLANE;
    }
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const unsigned long long i = i0 + 2 * k;
        const uint32_t lo = i < n ? codes[i] : 0u, hi = i + 1 < n ? codes[i + 1] : 0u;
        w[k] = lo | (hi << 16);
        cnt += (i < n) + (i + 1 < n);
    }
    return cnt;
}

__device__ __forceinline__ uint32_t code_at(const uint32_t w[16], int j) { return (w[j >> 1] >> (16 * (j & 1))) & 0xffffu; }

// ---- encode, pass 1: words per chunk, summed over each CTA's ENC_WARPS chunks
template <bool smem_tab>
__global__ void __launch_bounds__(ENC_THREADS) k_huff_sizes(const uint16_t *__restrict__ codes, unsigned long long n,
                                                           const uint8_t *__restrict__ lengths, int nsym, bool vec,
                                                           uint32_t *block_words, unsigned long long nchunks)
{
    extern __shared__ uint8_t len_sm[];  // nsym code lengths when they fit, else read from global memory
    __shared__ uint32_t warp_words[ENC_WARPS];
    if (smem_tab) {
        for (int i = threadIdx.x; i < nsym; i += ENC_THREADS) len_sm[i] = lengths[i];
        __syncthreads();
    }
    const uint8_t *len_s = smem_tab ? len_sm : lengths;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long chunk = (unsigned long long)blockIdx.x * ENC_WARPS + warp;
    uint32_t w[16];
    // past the last chunk the lane holds no codes (its first index is past n)
    const int cnt = lane_codes(codes, n, chunk * HCHUNK + (unsigned long long)lane * HLANE, vec, w);
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < HLANE; ++j)
        if (j < cnt) bits += len_s[code_at(w, j)];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, off);
    if (lane == 0) warp_words[warp] = (bits + 31) / 32;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < ENC_WARPS; ++k) sum += warp_words[k];
        block_words[blockIdx.x] = sum;
    }
    (void)nchunks;
}

// ---- one-CTA exclusive scan of the CTAs' word counts (in place); the total goes to *total
__global__ void __launch_bounds__(SCAN_THREADS) k_huff_scan(uint32_t *counts, unsigned long long m, uint32_t *total)
{
    constexpr int TILE = SCAN_THREADS * SCAN_ITEMS;
    __shared__ uint32_t tile[TILE];  // coalesced in and out; each thread scans SCAN_ITEMS consecutive entries
    __shared__ unsigned long long warp_sum[SCAN_THREADS / 32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    for (unsigned long long base = 0; base < m; base += TILE) {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const unsigned long long i = base + (unsigned long long)(k * SCAN_THREADS + tid);
            tile[k * SCAN_THREADS + tid] = i < m ? counts[i] : 0u;
        }
        __syncthreads();
        uint32_t v[SCAN_ITEMS];
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = tile[tid * SCAN_ITEMS + k];
        unsigned long long tsum = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) tsum += v[k];
        unsigned long long incl = tsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long ws = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, ws, off);
                if (lane >= off) ws += y;
            }
            warp_sum[lane] = ws;
        }
        __syncthreads();
        unsigned long long before = carry + (warp ? warp_sum[warp - 1] : 0ull) + incl - tsum;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            tile[tid * SCAN_ITEMS + k] = (uint32_t)before;
            before += v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const unsigned long long i = base + (unsigned long long)(k * SCAN_THREADS + tid);
            if (i < m) counts[i] = tile[k * SCAN_THREADS + tid];
        }
        if (tid == SCAN_THREADS - 1) carry = before;
        __syncthreads();
    }
    if (tid == 0) *total = (uint32_t)carry;
}

// ---- encode, pass 2: place the codewords
constexpr int MAX_WORDS = (HCHUNK * MAX_LEN + 31) / 32;  // words of a chunk at the longest codewords

template <bool smem_tab>
__global__ void __launch_bounds__(ENC_THREADS) k_huff_write(const uint16_t *__restrict__ codes, unsigned long long n,
                                                           const uint8_t *__restrict__ lengths,
                                                           const uint32_t *__restrict__ codewords, int nsym, bool vec,
                                                           const uint32_t *__restrict__ block_offset,
                                                           uint32_t *offsets, uint32_t *words,
                                                           unsigned long long nchunks,
                                                           unsigned long long capacity_words, unsigned int *bad)
{
    __shared__ uint32_t stage[ENC_WARPS * MAX_WORDS];
    __shared__ uint32_t warp_words[ENC_WARPS];
    extern __shared__ uint32_t tab_sm[];  // nsym codewords, then nsym lengths (bytes), when they fit
    const uint32_t *tab_s = codewords;
    const uint8_t *len_s = lengths;
    if (smem_tab) {
        uint8_t *l = reinterpret_cast<uint8_t *>(tab_sm + nsym);
        for (int i = threadIdx.x; i < nsym; i += ENC_THREADS) {
            tab_sm[i] = codewords[i];
            l[i] = lengths[i];
        }
        __syncthreads();
        tab_s = tab_sm;
        len_s = l;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long chunk = (unsigned long long)blockIdx.x * ENC_WARPS + warp;
    uint32_t w[16];
    const int cnt = lane_codes(codes, n, chunk * HCHUNK + (unsigned long long)lane * HLANE, vec, w);
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < HLANE; ++j)
        if (j < cnt) bits += len_s[code_at(w, j)];
    uint32_t pos = bits;  // inclusive, then exclusive scan of the lanes' bit counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pos, off);
        if (lane >= off) pos += y;
    }
    const uint32_t nw = (__shfl_sync(0xffffffffu, pos, 31) + 31) / 32;  // the chunk's words
    pos -= bits;
    if (lane == 0) warp_words[warp] = nw;
    __syncthreads();
    unsigned long long w0 = block_offset[blockIdx.x];
    for (int k = 0; k < warp; ++k) w0 += warp_words[k];
    if (chunk >= nchunks) return;  // whole warps leave together, after the CTA's barrier
    if (lane == 0) offsets[chunk] = (uint32_t)w0;
    uint32_t *sw = stage + warp * MAX_WORDS;
    if (nw > (uint32_t)MAX_WORDS || w0 + nw > capacity_words) {  // lengths above MAX_LEN,
        if (lane == 0) atomicOr(bad, 1u);                        // or too little room
        return;
    }
    for (uint32_t i = lane; i < nw; i += 32) sw[i] = 0u;
    __syncwarp();
    // accumulate the lane's bits MSB first from its start position; words wholly
    // inside the lane's range are stored, the first and last (shared with the
    // neighbouring lanes) are OR-ed in
    // (hi, lo) is a 64-bit shift register; its low nacc bits are pending (bits above them
    // are stale and never read: a word is taken from bits nacc-32 .. nacc-1)
    uint32_t hi = 0, lo = 0;
    uint32_t nacc = pos & 31;          // pending bits (the leading part of the first word is zero)
    uint32_t wi = pos >> 5;            // word being assembled
    const uint32_t first_word = wi;
#pragma unroll
    for (int j = 0; j < HLANE; ++j) {
        if (j >= cnt) break;
        const uint32_t c = code_at(w, j);
        const uint32_t len = len_s[c];  // 1..24
        hi = __funnelshift_l(lo, hi, len);
        lo = (lo << len) | tab_s[c];
        nacc += len;
        if (nacc >= 32) {  // a full word: pending bits nacc-32 .. nacc-1
            const uint32_t word = __funnelshift_r(lo, hi, nacc - 32);
            if (wi == first_word) atomicOr(&sw[wi], word);
            else sw[wi] = word;
            ++wi;
            nacc -= 32;
        }
    }
    if (nacc) atomicOr(&sw[wi], lo << (32 - nacc));  // nacc < 32: all pending bits are in lo
    __syncwarp();
    for (uint32_t i = lane; i < nw; i += 32) words[w0 + i] = sw[i];
}

// ---- decode tables from the lengths (one CTA): thread 0 lays out the canonical
// order (one pass over the symbols), then all threads fill the lookup table
__global__ void __launch_bounds__(TAB_THREADS) k_huff_tables(const uint8_t *__restrict__ lengths,
                                                             const uint32_t *__restrict__ codewords, int nsym,
                                                             DecodeTables *t, uint16_t *symbols, unsigned int *bad)
{
    constexpr int NL = MAX_LEN + 2, NW = TAB_THREADS / 32;
    __shared__ uint32_t cnt_s[NL], base_s[NL], run_s[NL];
    __shared__ uint32_t wcnt[NW][NL];  // per warp: symbols of each length, then their offset in the length's run
    __shared__ int maxl_s;
    __shared__ unsigned int bad_s;
    __shared__ uint32_t lut1[1 << LUT_BITS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < NL) {
        cnt_s[tid] = 0u;
        run_s[tid] = 0u;
        t->first[tid] = 0xffffffffu;
    }
    if (tid == 0) {
        maxl_s = 0;
        bad_s = 0u;
    }
    __syncthreads();
    // codewords per length
    for (int s = tid; s < nsym; s += TAB_THREADS) {
        const int l = lengths[s];
        if (l > MAX_LEN) {  // not a codebook this library builds
            bad_s = 1u;
        } else if (l) {
            atomicAdd(&cnt_s[l], 1u);
            atomicMax(&maxl_s, l);
        }
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t b = 0;
        for (int l = 0; l < NL; ++l) {
            base_s[l] = b;
            t->count[l] = cnt_s[l];
            t->base[l] = b;
            b += cnt_s[l];
        }
        t->max_len = maxl_s;
        *bad = bad_s;
    }
    __syncthreads();
    // canonical order: by length, ascending symbols within a length; TAB_THREADS symbols
    // at a time, ranked inside each warp, then across the warps, then after earlier rounds
    for (int s0 = 0; s0 < nsym; s0 += TAB_THREADS) {
        for (int i = tid; i < NW * NL; i += TAB_THREADS) (&wcnt[0][0])[i] = 0u;
        __syncthreads();
        const int s = s0 + tid;
        int l = s < nsym ? lengths[s] : 0;
        if (l > MAX_LEN) l = 0;
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (rank == 0) wcnt[warp][l] = (uint32_t)__popc(peers);
        __syncthreads();
        if (tid > 0 && tid < NL) {  // one thread per length: exclusive scan over the warps
            uint32_t acc = run_s[tid];
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            run_s[tid] = acc;
        }
        __syncthreads();
        if (l) {
            const uint32_t idx = base_s[l] + wcnt[warp][l] + (uint32_t)rank;
            symbols[idx] = (uint16_t)s;
            if (idx == base_s[l]) t->first[l] = codewords[s];
        }
        __syncthreads();
    }
    // one-codeword table (symbol << 8 | length, 0 = longer than LUT_BITS), then the
    // entries with every whole codeword of the LUT_BITS-bit window
    for (int i = tid; i < (1 << LUT_BITS); i += TAB_THREADS) lut1[i] = 0u;
    __syncthreads();
    for (int s = tid; s < nsym; s += TAB_THREADS) {
        const int l = lengths[s];
        if (!l || l > LUT_BITS) continue;
        const uint32_t lo = codewords[s] << (LUT_BITS - l), hi = lo + (1u << (LUT_BITS - l));
        for (uint32_t v = lo; v < hi && v < (1u << LUT_BITS); ++v) lut1[v] = ((uint32_t)s << 8) | (uint32_t)l;
    }
    __syncthreads();
    constexpr uint32_t MASK = (1u << LUT_BITS) - 1u;
    for (int v = tid; v < (1 << LUT_BITS); v += TAB_THREADS) {
        unsigned long long e = 0;
        uint32_t used = 0;
        int n = 0;
        for (; n < 3; ++n) {
            const uint32_t e1 = lut1[((uint32_t)v << used) & MASK];  // bits past the window read as 0
            const uint32_t l = e1 & 0xffu;
            if (!e1 || used + l > (uint32_t)LUT_BITS) break;  // not a whole codeword of the window
            used += l;
            e |= (unsigned long long)(e1 >> 8) << (16 * n);
            e |= (unsigned long long)used << (48 + 4 * n);
        }
        t->lut[v] = e | ((unsigned long long)n << 60);
    }
}

// ---- decode: one thread per chunk
__global__ void __launch_bounds__(DEC_THREADS) k_huff_decode(const uint32_t *__restrict__ words,
                                                            const uint32_t *__restrict__ offsets,
                                                            unsigned long long n, const DecodeTables *__restrict__ tg,
                                                            const uint16_t *__restrict__ symbols, int nsym_smem,
                                                            uint16_t *codes, unsigned long long nchunks, bool vec,
                                                            unsigned int *bad)
{
    __shared__ DecodeTables t;
    __shared__ uint32_t stage[DEC_THREADS * (DEC_ROUND / 2 + 1)];  // a row of DEC_ROUND codes per thread, padded
    extern __shared__ uint16_t sym_s[];  // the symbol list when it fits (nsym_smem)
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tg);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&t);
        for (int i = threadIdx.x; i < (int)(sizeof(DecodeTables) / 4); i += DEC_THREADS) dst[i] = src[i];
        for (int i = threadIdx.x; i < nsym_smem; i += DEC_THREADS) sym_s[i] = symbols[i];
    }
    __syncthreads();
    const uint16_t *sym_tab = nsym_smem ? sym_s : symbols;
    constexpr int RW = DEC_ROUND / 2 + 1;  // row pitch in words: thread rows fall in distinct banks
    const int lane = threadIdx.x & 31;
    const unsigned long long chunk = (unsigned long long)blockIdx.x * DEC_THREADS + threadIdx.x;
    const unsigned long long chunk0 = chunk - lane;  // the warp's first chunk
    if (chunk0 >= nchunks) return;                  // whole warps leave together
    const bool live = chunk < nchunks;
    const uint32_t *w = words;
    uint32_t nw = 0;
    if (live) {
        w = words + offsets[chunk];
        nw = offsets[chunk + 1] - offsets[chunk];
    }
    // 64-bit window: the next 64 bits of the chunk, left-aligned; the word after it is
    // loaded one refill ahead of its use
    unsigned long long win = ((unsigned long long)(nw > 0 ? w[0] : 0u) << 32) | (nw > 1 ? w[1] : 0u);
    uint32_t ahead = nw > 2 ? w[2] : 0u;
    uint32_t next = 3;    // next word to take
    int avail = 64;       // valid bits in win (beyond the chunk's words they are zeros)
    const int cnt = live ? (int)min((unsigned long long)HCHUNK, n - chunk * HCHUNK) : 0;
    const int maxl = t.max_len;
    bool ok = true;
    uint16_t *row = reinterpret_cast<uint16_t *>(stage + threadIdx.x * RW);
    const uint32_t *wrows = stage + (threadIdx.x - lane) * RW;
    // the warp's 32 chunks all hold HCHUNK codes and the codes are 4-byte aligned: the
    // store phase needs no checks; each lane stores the words 2*(lane&15), +1 of row
    // r + (lane >> 4) through a running pointer
    const bool fast_store = vec && (chunk0 + 32) * HCHUNK <= n;
    uint32_t *store_base = reinterpret_cast<uint32_t *>(codes + (chunk0 + (lane >> 4)) * HCHUNK) + (lane & 15);
    for (int j0 = 0; j0 < HCHUNK; j0 += DEC_ROUND) {
        const int jn = ok ? min(DEC_ROUND, cnt - j0) : 0;
        int j = 0;
        while (j < jn) {
            const uint32_t top = (uint32_t)(win >> 32);
            const unsigned long long e = t.lut[top >> (32 - LUT_BITS)];
            const int ne = (int)(e >> 60);
            uint32_t len;
            if (ne) {  // up to three whole codewords; take what the round still needs
                const int take = min(ne, jn - j);
                row[j] = (uint16_t)e;
                if (take > 1) row[j + 1] = (uint16_t)(e >> 16);
                if (take > 2) row[j + 2] = (uint16_t)(e >> 32);
                len = (uint32_t)(e >> (48 + 4 * (take - 1))) & 0xfu;
                j += take;
            } else {  // longer codeword: the canonical rule, length by length
                len = 0;
                uint32_t sym = 0;
                for (int l = LUT_BITS + 1; l <= maxl; ++l) {
                    const uint32_t v = top >> (32 - l);
                    if (t.count[l] && v >= t.first[l] && v - t.first[l] < t.count[l]) {
                        sym = sym_tab[t.base[l] + (v - t.first[l])];
                        len = (uint32_t)l;
                        break;
                    }
                }
                if (!len) {  // not a codeword: corrupt stream; the thread stays for its warp's stores
                    atomicOr(bad, 1u);
                    ok = false;
                    break;
                }
                row[j++] = (uint16_t)sym;
            }
            win <<= len;
            avail -= (int)len;
            if (avail <= 32) {  // refill the low 32 bits
                win |= (unsigned long long)ahead << (32 - avail);
                avail += 32;
                ahead = next < nw ? w[next] : 0u;
                ++next;
            }
        }
        __syncwarp();
        // the warp stores its 32 rows of this round, two rows (2 x DEC_ROUND codes) per instruction
        static_assert(DEC_ROUND == 32, "two staged rows per warp store");
        if (fast_store) {  // 32 whole chunks, 4-byte aligned codes: no checks, running pointers
            uint32_t *dst = store_base + (j0 >> 1);
            const uint32_t *src = wrows + (lane >> 4) * RW + (lane & 15);
#pragma unroll 4
            for (int r = 0; r < 32; r += 2) dst[(size_t)r * (HCHUNK / 2)] = src[r * RW];
        } else {
            for (int r = 0; r < 32; r += 2) {
                const int rr = r + (lane >> 4), e = 2 * (lane & 15);
                const unsigned long long c = chunk0 + rr;
                if (c >= nchunks) break;
                const long long m = min((long long)DEC_ROUND,
                                        (long long)min((unsigned long long)HCHUNK, n - c * HCHUNK) - j0);  // codes to store
                if (m <= 0) continue;
                uint16_t *dst = codes + c * HCHUNK + j0;
                const uint32_t v = wrows[rr * RW + (lane & 15)];
                if (vec && e + 1 < m) {
                    *reinterpret_cast<uint32_t *>(dst + e) = v;
                } else {
                    if (e < m) dst[e] = (uint16_t)(v & 0xffffu);
                    if (e + 1 < m) dst[e + 1] = (uint16_t)(v >> 16);
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace

unsigned long long huffman_chunks(unsigned long long n) { return (n + HCHUNK - 1) / HCHUNK; }

unsigned long long huffman_capacity_words(unsigned long long n, int max_len)
{
    return huffman_chunks(n) * (unsigned long long)((HCHUNK * max_len + 31) / 32);
}

size_t huffman_decode_workspace(int nsym)
{
    return ((sizeof(DecodeTables) + 15) / 16) * 16 + sizeof(uint16_t) * (size_t)nsym + 16;
}

int huffman_max_len() { return MAX_LEN; }

// Host: code lengths by Huffman's construction (ties by weight, then creation
// order: symbols by index, merged nodes after) limited to max_len (lengths above
// it are cut to max_len, then the longest codewords below it are lengthened until
// the Kraft sum is at most 1), and canonical codewords.
bool huffman_codebook(const uint32_t *hist, int nsym, int max_len, uint8_t *lengths, uint32_t *codewords)
{
    if (max_len < 1 || max_len > MAX_LEN) return false;
    std::vector<int> used;
    for (int s = 0; s < nsym; ++s) {
        lengths[s] = 0;
        codewords[s] = 0;
        if (hist[s]) used.push_back(s);
    }
    if (used.empty()) return true;
    if (used.size() > (size_t(1) << max_len)) return false;  // no prefix code of max_len bits holds them
    std::vector<int> len(nsym, 0);
    if (used.size() == 1) {
        len[used[0]] = 1;
    } else {
        // nodes: leaves 0..nsym-1 (by symbol), internal nodes nsym.. in creation order
        std::vector<int> parent(2 * nsym, -1);
        using Item = std::pair<unsigned long long, int>;  // (weight, node id): smallest first
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
        for (int s : used) pq.push({hist[s], s});
        int next = nsym;
        while (pq.size() > 1) {
            const Item a = pq.top();
            pq.pop();
            const Item b = pq.top();
            pq.pop();
            parent[a.second] = next;
            parent[b.second] = next;
            pq.push({a.first + b.first, next});
            ++next;
        }
        for (int s : used) {
            int d = 0;
            for (int v = s; parent[v] >= 0; v = parent[v]) ++d;
            len[s] = d;
        }
    }
    // length limit
    int longest = 0;
    for (int s : used) longest = std::max(longest, len[s]);
    if (longest > max_len) {
        unsigned long long kraft = 0;  // in units of 2^-max_len
        for (int s : used) {
            len[s] = std::min(len[s], max_len);
            kraft += 1ull << (max_len - len[s]);
        }
        while (kraft > (1ull << max_len)) {
            int pick = -1;
            for (int s : used) {
                if (len[s] >= max_len) continue;
                if (pick < 0 || len[s] > len[pick] || (len[s] == len[pick] && hist[s] < hist[pick]) ||
                    (len[s] == len[pick] && hist[s] == hist[pick] && s > pick))
                    pick = s;
            }
            kraft -= 1ull << (max_len - len[pick] - 1);
            ++len[pick];
        }
    }
    // canonical codewords: by (length, symbol)
    std::vector<std::pair<int, int>> order;
    for (int s : used) order.push_back({len[s], s});
    std::sort(order.begin(), order.end());
    uint32_t code = 0;
    int prev = order.front().first;
    for (const auto &p : order) {
        code <<= (p.first - prev);
        codewords[p.second] = code;
        lengths[p.second] = (uint8_t)p.first;
        ++code;
        prev = p.first;
    }
    return true;
}

size_t huffman_encode_workspace(unsigned long long n)
{
    const unsigned long long blocks = (huffman_chunks(n) + ENC_WARPS - 1) / ENC_WARPS;
    return ((4 * blocks + 255) / 256) * 256;
}

cudaError_t launch_huffman_encode(const uint16_t *codes, unsigned long long n, const uint8_t *lengths,
                                  const uint32_t *codewords, int nsym, uint32_t *offsets, uint32_t *words,
                                  unsigned long long capacity_words, uint32_t *block_words, unsigned int *bad,
                                  cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const unsigned long long nch = huffman_chunks(n);
    if (nch == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
    const unsigned long long blocks = (nch + ENC_WARPS - 1) / ENC_WARPS;
    const bool vec = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
    // the codebook sits in shared memory up to 16384 symbols (80 KB), beyond that it is
    // read through the cache
    const bool smem_tab = nsym <= 16384;
    const size_t tab = 5 * (size_t)nsym;  // codewords + lengths
    if (smem_tab) {
        if (tab > 40 * 1024) {
            e = cudaFuncSetAttribute(k_huff_sizes<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, nsym);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_huff_write<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
            if (e != cudaSuccess) return e;
        }
        k_huff_sizes<true><<<(unsigned)blocks, ENC_THREADS, nsym, s>>>(codes, n, lengths, nsym, vec, block_words,
                                                                       nch);
    } else {
        k_huff_sizes<false><<<(unsigned)blocks, ENC_THREADS, 0, s>>>(codes, n, lengths, nsym, vec, block_words, nch);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_huff_scan<<<1, SCAN_THREADS, 0, s>>>(block_words, blocks, offsets + nch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (smem_tab)
        k_huff_write<true><<<(unsigned)blocks, ENC_THREADS, tab, s>>>(codes, n, lengths, codewords, nsym, vec,
                                                                      block_words, offsets, words, nch,
                                                                      capacity_words, bad);
    else
        k_huff_write<false><<<(unsigned)blocks, ENC_THREADS, 0, s>>>(codes, n, lengths, codewords, nsym, vec,
                                                                     block_words, offsets, words, nch,
                                                                     capacity_words, bad);
    return cudaGetLastError();
}

cudaError_t launch_huffman_decode(const uint32_t *words, const uint32_t *offsets, unsigned long long n,
                                  const uint8_t *lengths, const uint32_t *codewords, int nsym, uint16_t *codes,
                                  void *ws, unsigned int *bad, cudaStream_t s)
{
    DecodeTables *t = static_cast<DecodeTables *>(ws);
    uint16_t *symbols =
        reinterpret_cast<uint16_t *>(static_cast<unsigned char *>(ws) + ((sizeof(DecodeTables) + 15) / 16) * 16);
    k_huff_tables<<<1, TAB_THREADS, 0, s>>>(lengths, codewords, nsym, t, symbols, bad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned long long nch = huffman_chunks(n);
    if (nch == 0) return cudaSuccess;
    const bool vec = (reinterpret_cast<uintptr_t>(codes) & 3u) == 0;
    const int nsym_smem = nsym <= SYM_SMEM ? nsym : 0;
    const size_t dyn = 2 * (size_t)nsym_smem;
    k_huff_decode<<<(unsigned)((nch + DEC_THREADS - 1) / DEC_THREADS), DEC_THREADS, dyn, s>>>(
        words, offsets, n, t, symbols, nsym_smem, codes, nch, vec, bad);
    return cudaGetLastError();
}

}  // namespace gi
