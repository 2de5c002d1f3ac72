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
// Encoding: one warp per chunk, each lane 32 consecutive codes.  A first pass
// sums the code lengths per chunk, a one-CTA scan turns them into word offsets,
// and a second pass has every lane place its codewords at its bit offset (a
// warp scan) in the warp's shared-memory copy of the chunk, which is then
// written out with coalesced stores.
// Decoding: one thread per chunk, reading its words in order: the first 11 bits
// index a lookup table (symbol, length); longer codewords take the canonical
// rule (per length, the first codeword and the first symbol index).
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
constexpr int LUT_BITS = 11;
constexpr int SCAN_THREADS = 1024;
constexpr int DEC_THREADS = 128;

// Device decode tables, built per call from the code lengths.
struct DecodeTables {
    uint32_t first[MAX_LEN + 2];      // first codeword of each length (canonical)
    uint32_t count[MAX_LEN + 2];      // codewords of each length
    uint32_t base[MAX_LEN + 2];       // index in `symbols` of each length's first symbol
    uint32_t lut[1 << LUT_BITS];      // (symbol << 8) | length for codewords of <= LUT_BITS bits; 0 = longer
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

// ---- encode, pass 1: bits per chunk -> words per chunk
__global__ void __launch_bounds__(ENC_THREADS) k_huff_sizes(const uint16_t *__restrict__ codes, unsigned long long n,
                                                           const uint8_t *__restrict__ lengths, int nsym, bool vec,
                                                           uint32_t *chunk_words, unsigned long long nchunks)
{
    extern __shared__ uint8_t len_s[];  // nsym code lengths
    for (int i = threadIdx.x; i < nsym; i += ENC_THREADS) len_s[i] = lengths[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long chunk = (unsigned long long)blockIdx.x * ENC_WARPS + (threadIdx.x >> 5);
    if (chunk >= nchunks) return;
    uint32_t w[16];
    const int cnt = lane_codes(codes, n, chunk * HCHUNK + (unsigned long long)lane * HLANE, vec, w);
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < HLANE; ++j)
        if (j < cnt) bits += len_s[code_at(w, j)];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, off);
    if (lane == 0) chunk_words[chunk] = (bits + 31) / 32;
}

// ---- one-CTA exclusive scan of the chunk word counts (in place, total appended)
__global__ void __launch_bounds__(SCAN_THREADS) k_huff_scan(uint32_t *offsets, unsigned long long nchunks)
{
    __shared__ unsigned long long warp_sum[SCAN_THREADS / 32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (unsigned long long base = 0; base < nchunks; base += SCAN_THREADS) {
        const unsigned long long i = base + threadIdx.x;
        const unsigned long long v = i < nchunks ? offsets[i] : 0u;
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
            warp_sum[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? warp_sum[warp - 1] : 0ull) + incl - v;
        if (i < nchunks) offsets[i] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[nchunks] = (uint32_t)carry;
}

// ---- encode, pass 2: place the codewords
constexpr int MAX_WORDS = (HCHUNK * MAX_LEN + 31) / 32;  // words of a chunk at the longest codewords

__global__ void __launch_bounds__(ENC_THREADS) k_huff_write(const uint16_t *__restrict__ codes, unsigned long long n,
                                                           const uint8_t *__restrict__ lengths,
                                                           const uint32_t *__restrict__ codewords, int nsym, bool vec,
                                                           const uint32_t *__restrict__ offsets, uint32_t *words,
                                                           unsigned long long nchunks,
                                                           unsigned long long capacity_words, unsigned int *bad)
{
    __shared__ uint32_t stage[ENC_WARPS * MAX_WORDS];
    extern __shared__ uint32_t tab_s[];  // nsym codewords, then nsym lengths (bytes)
    uint8_t *len_s = reinterpret_cast<uint8_t *>(tab_s + nsym);
    for (int i = threadIdx.x; i < nsym; i += ENC_THREADS) {
        tab_s[i] = codewords[i];
        len_s[i] = lengths[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long chunk = (unsigned long long)blockIdx.x * ENC_WARPS + warp;
    if (chunk >= nchunks) return;  // whole warps leave together
    uint32_t *sw = stage + warp * MAX_WORDS;
    const uint32_t w0 = offsets[chunk], nw = offsets[chunk + 1] - w0;
    if (nw > (uint32_t)MAX_WORDS || (unsigned long long)w0 + nw > capacity_words) {  // lengths above MAX_LEN,
        if (lane == 0) atomicOr(bad, 1u);                                             // or too little room
        return;
    }
    for (uint32_t i = lane; i < nw; i += 32) sw[i] = 0u;
    __syncwarp();
    uint32_t w[16];
    const int cnt = lane_codes(codes, n, chunk * HCHUNK + (unsigned long long)lane * HLANE, vec, w);
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < HLANE; ++j)
        if (j < cnt) bits += len_s[code_at(w, j)];
    uint32_t pos = bits;  // exclusive scan of the lanes' bit counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pos, off);
        if (lane >= off) pos += y;
    }
    pos -= bits;
    // accumulate the lane's bits MSB first from its start position; words wholly
    // inside the lane's range are stored, the first and last (shared with the
    // neighbouring lanes) are OR-ed in
    unsigned long long acc = 0;
    uint32_t nacc = pos & 31;          // bits already in acc (the leading part of the first word is zero)
    uint32_t wi = pos >> 5;            // word being assembled
    const uint32_t first_word = wi;
#pragma unroll
    for (int j = 0; j < HLANE; ++j) {
        if (j >= cnt) break;
        const uint32_t c = code_at(w, j);
        const uint32_t len = len_s[c];
        acc = (acc << len) | tab_s[c];
        nacc += len;
        if (nacc >= 32) {  // a full word: its top 32 bits
            const uint32_t word = (uint32_t)(acc >> (nacc - 32));
            if (wi == first_word) atomicOr(&sw[wi], word);
            else sw[wi] = word;
            ++wi;
            nacc -= 32;
            acc &= (nacc ? ((1ull << nacc) - 1ull) : 0ull);
        }
    }
    if (nacc) atomicOr(&sw[wi], (uint32_t)(acc << (32 - nacc)));
    __syncwarp();
    for (uint32_t i = lane; i < nw; i += 32) words[w0 + i] = sw[i];
}

// ---- decode tables from the lengths (one CTA): thread 0 lays out the canonical
// order (one pass over the symbols), then all threads fill the lookup table
__global__ void k_huff_tables(const uint8_t *__restrict__ lengths, const uint32_t *__restrict__ codewords, int nsym,
                              DecodeTables *t, uint16_t *symbols, unsigned int *bad)
{
    for (int i = threadIdx.x; i < (1 << LUT_BITS); i += blockDim.x) t->lut[i] = 0u;
    if (threadIdx.x == 0) {
        *bad = 0u;
        uint32_t cnt[MAX_LEN + 2] = {0};
        int maxl = 0;
        for (int s = 0; s < nsym; ++s) {
            int l = lengths[s];
            if (l > MAX_LEN) {  // not a codebook this library builds
                *bad = 1u;
                l = 0;
            }
            if (l) {
                ++cnt[l];
                maxl = max(maxl, l);
            }
        }
        uint32_t base = 0, nextidx[MAX_LEN + 2];
        for (int l = 0; l <= MAX_LEN + 1; ++l) {
            t->count[l] = cnt[l];
            t->base[l] = base;
            t->first[l] = 0xffffffffu;
            nextidx[l] = base;
            base += cnt[l];
        }
        t->max_len = maxl;
        for (int s = 0; s < nsym; ++s) {  // ascending symbols: canonical order within each length
            const int l = lengths[s];
            if (!l || l > MAX_LEN) continue;
            if (nextidx[l] == t->base[l]) t->first[l] = codewords[s];
            symbols[nextidx[l]++] = (uint16_t)s;
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nsym; s += blockDim.x) {
        const int l = lengths[s];
        if (!l || l > LUT_BITS) continue;
        const uint32_t lo = codewords[s] << (LUT_BITS - l), hi = lo + (1u << (LUT_BITS - l));
        for (uint32_t v = lo; v < hi && v < (1u << LUT_BITS); ++v) t->lut[v] = ((uint32_t)s << 8) | (uint32_t)l;
    }
}

// ---- decode: one thread per chunk
__global__ void __launch_bounds__(DEC_THREADS) k_huff_decode(const uint32_t *__restrict__ words,
                                                            const uint32_t *__restrict__ offsets,
                                                            unsigned long long n, const DecodeTables *__restrict__ tg,
                                                            const uint16_t *__restrict__ symbols, uint16_t *codes,
                                                            unsigned long long nchunks, bool vec, unsigned int *bad)
{
    __shared__ DecodeTables t;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tg);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&t);
        for (int i = threadIdx.x; i < (int)(sizeof(DecodeTables) / 4); i += DEC_THREADS) dst[i] = src[i];
    }
    __syncthreads();
    const unsigned long long chunk = (unsigned long long)blockIdx.x * DEC_THREADS + threadIdx.x;
    if (chunk >= nchunks) return;
    const uint32_t *w = words + offsets[chunk];
    const uint32_t nw = offsets[chunk + 1] - offsets[chunk];
    // 64-bit window: the next 64 bits of the chunk, left-aligned
    unsigned long long win = ((unsigned long long)(nw > 0 ? w[0] : 0u) << 32) | (nw > 1 ? w[1] : 0u);
    uint32_t next = 2;    // next word to load
    int avail = 64;       // valid bits in win (beyond the chunk's words they are zeros)
    const unsigned long long i0 = chunk * HCHUNK;
    const int cnt = (int)min((unsigned long long)HCHUNK, n - i0);
    const int maxl = t.max_len;
    uint32_t ob[4] = {0u, 0u, 0u, 0u};
    for (int j = 0; j < cnt; ++j) {
        const uint32_t top = (uint32_t)(win >> 32);
        uint32_t e = t.lut[top >> (32 - LUT_BITS)];
        uint32_t sym, len;
        if (e) {
            sym = e >> 8;
            len = e & 0xffu;
        } else {  // longer codeword: the canonical rule, length by length
            len = 0;
            sym = 0;
            for (int l = LUT_BITS + 1; l <= maxl; ++l) {
                const uint32_t v = top >> (32 - l);
                if (t.count[l] && v >= t.first[l] && v - t.first[l] < t.count[l]) {
                    sym = symbols[t.base[l] + (v - t.first[l])];
                    len = (uint32_t)l;
                    break;
                }
            }
            if (!len) {  // not a codeword: corrupt stream
                atomicOr(bad, 1u);
                return;
            }
        }
        // eight codes per 16-byte store (the chunk starts 2048-byte aligned)
        ob[(j & 7) >> 1] |= sym << (16 * (j & 1));
        if ((j & 7) == 7) {
            if (vec) {
                *reinterpret_cast<uint4 *>(codes + i0 + j - 7) = make_uint4(ob[0], ob[1], ob[2], ob[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) codes[i0 + j - 7 + k] = (uint16_t)(ob[k >> 1] >> (16 * (k & 1)));
            }
            ob[0] = ob[1] = ob[2] = ob[3] = 0u;
        }
        win <<= len;
        avail -= (int)len;
        if (avail <= 32) {  // refill the low 32 bits
            const uint32_t nxt = next < nw ? w[next] : 0u;
            win |= (unsigned long long)nxt << (32 - avail);
            avail += 32;
            ++next;
        }
    }
    for (int k = cnt & ~7; k < cnt; ++k) codes[i0 + k] = (uint16_t)(ob[(k & 7) >> 1] >> (16 * (k & 1)));
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

cudaError_t launch_huffman_encode(const uint16_t *codes, unsigned long long n, const uint8_t *lengths,
                                  const uint32_t *codewords, int nsym, uint32_t *offsets, uint32_t *words,
                                  unsigned long long capacity_words, unsigned int *bad, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const unsigned long long nch = huffman_chunks(n);
    if (nch == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
    const unsigned long long blocks = (nch + ENC_WARPS - 1) / ENC_WARPS;
    const bool vec = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
    k_huff_sizes<<<(unsigned)blocks, ENC_THREADS, nsym, s>>>(codes, n, lengths, nsym, vec, offsets, nch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_huff_scan<<<1, SCAN_THREADS, 0, s>>>(offsets, nch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t tab = 5 * (size_t)nsym;  // codewords + lengths
    if (tab > 40 * 1024) {
        e = cudaFuncSetAttribute(k_huff_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
        if (e != cudaSuccess) return e;
    }
    k_huff_write<<<(unsigned)blocks, ENC_THREADS, tab, s>>>(codes, n, lengths, codewords, nsym, vec, offsets, words,
                                                            nch, capacity_words, bad);
    return cudaGetLastError();
}

cudaError_t launch_huffman_decode(const uint32_t *words, const uint32_t *offsets, unsigned long long n,
                                  const uint8_t *lengths, const uint32_t *codewords, int nsym, uint16_t *codes,
                                  void *ws, unsigned int *bad, cudaStream_t s)
{
    DecodeTables *t = static_cast<DecodeTables *>(ws);
    uint16_t *symbols =
        reinterpret_cast<uint16_t *>(static_cast<unsigned char *>(ws) + ((sizeof(DecodeTables) + 15) / 16) * 16);
    k_huff_tables<<<1, 1024, 0, s>>>(lengths, codewords, nsym, t, symbols, bad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned long long nch = huffman_chunks(n);
    if (nch == 0) return cudaSuccess;
    const bool vec = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
    k_huff_decode<<<(unsigned)((nch + DEC_THREADS - 1) / DEC_THREADS), DEC_THREADS, 0, s>>>(words, offsets, n, t,
                                                                                           symbols, codes, nch, vec,
                                                                                           bad);
    return cudaGetLastError();
}

}  // namespace gi
