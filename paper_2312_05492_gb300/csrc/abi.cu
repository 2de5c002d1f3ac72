// C ABI of libginterp.so (declared in include/ginterp.h): argument checks,
// workspace layout and the stream-ordered launch sequences of compression
// (profile -> range/bounds -> tiles -> outlier compaction) and decompression
// (outlier scatter -> tiles).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gi {
size_t range_partials_bytes();
}

namespace {

using gi::Dims;

constexpr size_t kAlign = 256;
constexpr size_t kCtrlBytes = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool dims_ok(const int64_t *dims)
{
    if (!dims) return false;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t)0x7fffffff) return false;
    const double n = (double)dims[0] * (double)dims[1] * (double)dims[2];
    return n < 4294967296.0;  // u32 outlier indices
}

bool cfg_ok(const interp_config *c)
{
    if (!c) return false;
    int seen = 0;
    for (int a = 0; a < 3; ++a) {
        if (c->dim_order[a] < 0 || c->dim_order[a] > 2) return false;
        seen |= 1 << c->dim_order[a];
        if (c->level_kind[a] != 0 && c->level_kind[a] != 1) return false;
        if (c->cubic_kind[a] != 0 && c->cubic_kind[a] != 1) return false;
    }
    if (seen != 7) return false;
    if (c->eb_mode != 0 && c->eb_mode != 1) return false;
    if (c->domain_x != 0 && c->domain_x != 8 && c->domain_x != 32) return false;
    if (c->ndim < 0 || c->ndim > 3) return false;
    if (c->ndim == 1 || c->ndim == 2) {
        if (c->domain_x == 32) return false;
    }
    if (c->autotune != 0 && c->autotune != 1) return false;
    if (c->radius < 2 || c->radius > 32768) return false;
    if (std::isnan(c->alpha) || std::isinf(c->alpha)) return false;
    return true;
}

// outlier bitmap: one word per 32 x-positions of every row; the counters are
// per 2048 words in ascending index order, the words themselves are stored
// tile-major (see tiles.cu)
Dims to_dims(const int64_t *d) { return Dims{(int)d[0], (int)d[1], (int)d[2]}; }

int64_t bitmap_words(const int64_t *dims) { return dims[0] * dims[1] * ((dims[2] + 31) / 32); }

struct WsLayout {
    size_t ctrl, partials, bitmap, blockcnt, total;
    int64_t words;
    int nblk;
};

WsLayout ws_layout(const int64_t *dims)
{
    WsLayout L;
    L.words = bitmap_words(dims);
    L.nblk = (int)((L.words + gi::BITMAP_BLOCK_WORDS - 1) / gi::BITMAP_BLOCK_WORDS);
    L.ctrl = 0;
    L.partials = kCtrlBytes;
    L.bitmap = align_up(L.partials + gi::range_partials_bytes());
    L.blockcnt = align_up(L.bitmap + sizeof(uint32_t) * gi::bitmap_words_tiled(to_dims(dims)));
    L.total = align_up(L.blockcnt + sizeof(uint32_t) * (size_t)L.nblk);
    return L;
}

// Eq. 1 (Sec. IV-B.2): alpha = A(eps), piecewise linear in the relative bound.
double alpha_of_eps(double eps)
{
    if (eps >= 1e-1) return 2.0;
    if (eps >= 1e-2) return 1.75 + 0.25 * (eps - 1e-2) / (1e-1 - 1e-2);
    if (eps >= 1e-3) return 1.5 + 0.25 * (eps - 1e-3) / (1e-2 - 1e-3);
    if (eps >= 1e-4) return 1.25 + 0.25 * (eps - 1e-4) / (1e-3 - 1e-4);
    if (eps >= 1e-5) return 1.0 + 0.25 * (eps - 1e-5) / (1e-4 - 1e-5);
    return 1.0;
}

double effective_alpha(const interp_config &c, double eb)
{
    if (c.alpha > 0) return c.alpha;
    return c.eb_mode ? alpha_of_eps(eb) : 1.0;
}

// Codes per store for rows of 8 codes starting at multiples of 8 along x: the
// widest store whose alignment every such row start keeps.
int code_store_width(const void *codes, int nx)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(codes);
    if (a % 16 == 0 && nx % 8 == 0) return 8;
    if (a % 8 == 0 && nx % 4 == 0) return 4;
    if (a % 4 == 0 && nx % 2 == 0) return 2;
    return 1;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? INTERP_OK : INTERP_ECUDA; }

// ---- optional event timing around the tile kernels (measurement only)
constexpr int kTimingPairs = 512;
struct TimingLog {
    cudaEvent_t ev[2][kTimingPairs][2];
    int used[2];
    bool created;
    bool on;
};
TimingLog g_timing{};

void timing_mark(int kind, int edge, cudaStream_t s)
{
    if (!g_timing.on) return;
    const int i = g_timing.used[kind];
    if (i >= kTimingPairs) return;
    cudaEventRecord(g_timing.ev[kind][i][edge], s);
    if (edge == 1) g_timing.used[kind] = i + 1;
}

}  // namespace

extern "C" {

size_t interp_anchor_count(const int64_t dims[3])
{
    if (!dims_ok(dims)) return 0;
    size_t n = 1;
    for (int a = 0; a < 3; ++a) n *= (size_t)((dims[a] - 1) / 8 + 1);
    return n;
}

size_t interp_anchor_count_nd(const int64_t dims[3], int32_t ndim)
{
    if (!dims_ok(dims) || ndim < 0 || ndim > 3) return 0;
    if (ndim == 0 || ndim == 3) return interp_anchor_count(dims);
    const int64_t edge = ndim == 2 ? 16 : 512;
    size_t n = 1;
    for (int a = 0; a < 3; ++a) n *= (size_t)((dims[a] - 1) / (a >= 3 - ndim ? edge : 1) + 1);
    return n;
}

size_t interp_workspace_bytes(const int64_t dims[3], const interp_config *cfg)
{
    if (!dims_ok(dims) || !cfg_ok(cfg)) return 0;
    return ws_layout(dims).total;
}

// The compression set-up of one field (zeroing, profile, range and bounds).
// The 1-D / 2-D chunk geometries (interp_config.ndim 1 or 2); 0 and 3 are 3-D.
bool is_nd(int32_t ndim) { return ndim == 1 || ndim == 2; }

gi::PrologueItem prologue_item(const interp_compress_item &it, const WsLayout &L)
{
    unsigned char *ws = static_cast<unsigned char *>(it.d_ws);
    gi::PrologueItem p;
    p.x = it.d_x;
    p.d = to_dims(it.dims);
    p.eb = it.eb;
    p.cfg = it.cfg;
    p.alpha = effective_alpha(it.cfg, it.eb);
    p.hdr = it.d_hdr;
    p.counter = reinterpret_cast<uint32_t *>(ws + L.ctrl);
    p.ctrl_words = (int)(kCtrlBytes / sizeof(uint32_t));
    p.partials = ws + L.partials;
    p.blockcnt = reinterpret_cast<uint32_t *>(ws + L.blockcnt);
    p.nblk = L.nblk;
    p.hist = it.d_hist;
    return p;
}

// One field in the 1-D or 2-D geometry: the same setup and compaction as the 3-D
// path around the per-tile kernel of nd.cu.
int compress_nd(const interp_compress_item &it, interp_stream_t stream)
{
    const interp_config &c = it.cfg;
    if (!dims_ok(it.dims) || !cfg_ok(&c)) return INTERP_EINVAL;
    if (!(it.eb > 0.0) || std::isinf(it.eb)) return INTERP_EINVAL;
    if (!it.d_x || !it.d_anchors || !it.d_codes || !it.d_hdr || !it.d_ws) return INTERP_EINVAL;
    if (it.out_capacity > 0 && (!it.d_out_idx || !it.d_out_val)) return INTERP_EINVAL;
    const WsLayout L = ws_layout(it.dims);
    if (it.ws_bytes < L.total) return INTERP_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Dims d = to_dims(it.dims);
    const double alpha = effective_alpha(c, it.eb);
    unsigned char *ws = static_cast<unsigned char *>(it.d_ws);
    unsigned int *counter = reinterpret_cast<unsigned int *>(ws + L.ctrl);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(ws + L.bitmap);
    uint32_t *blockcnt = reinterpret_cast<uint32_t *>(ws + L.blockcnt);
    (void)counter;
    (void)alpha;
    const gi::PrologueItem pro = prologue_item(it, L);
    cudaError_t e = gi::launch_prologue(&pro, 1, s);
    const gi::CompressArgs args{it.d_x, d, it.d_anchors, it.d_codes, bitmap, blockcnt, it.d_hist, c.radius,
                                it.d_hdr, false, false, 1};
    if (e == cudaSuccess) {
        timing_mark(0, 0, s);
        e = gi::launch_nd_compress(c.ndim, args, s);
        timing_mark(0, 1, s);
    }
    if (e == cudaSuccess) {
        // row-major bitmap (nd.cu); the 1-D / 2-D kernels count every bin themselves
        const gi::CompactItem ci{bitmap, blockcnt, L.words, d, it.d_x, it.d_out_idx, it.d_out_val,
                                 it.out_capacity, it.d_hdr, true, nullptr, c.radius};
        e = gi::launch_outlier_compaction(&ci, 1, s);
    }
    return cuda_status(e);
}

int interp_compress_batched(const interp_compress_item *items, int n, interp_stream_t stream)
{
    return interp_compress_batched_scheduled(items, n, nullptr, stream);
}

int interp_compress_batched_scheduled(const interp_compress_item *items, int n, const interp_tile_schedule *sched,
                                      interp_stream_t stream)
{
    if (sched && (sched->run < 0 || sched->ctas_per_sm < 0)) return INTERP_EINVAL;
    if (!items || n < 1 || n > gi::kMaxBatch) return INTERP_EINVAL;
    WsLayout L[gi::kMaxBatch];
    for (int i = 0; i < n; ++i) {  // every argument is checked before anything is enqueued
        const interp_compress_item &it = items[i];
        if (!dims_ok(it.dims) || !cfg_ok(&it.cfg)) return INTERP_EINVAL;
        if (!(it.eb > 0.0) || std::isinf(it.eb)) return INTERP_EINVAL;
        if (!it.d_x || !it.d_anchors || !it.d_codes || !it.d_hdr || !it.d_ws) return INTERP_EINVAL;
        if (it.out_capacity > 0 && (!it.d_out_idx || !it.d_out_val)) return INTERP_EINVAL;
        L[i] = ws_layout(it.dims);
        if (it.ws_bytes < L[i].total) return INTERP_EWORKSPACE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // set-up of every field in two launches (zeroing; profile, range and bounds)
    gi::CompressArgs args[gi::kMaxBatch], args3[gi::kMaxBatch];
    gi::PrologueItem pro[gi::kMaxBatch];
    int n3 = 0;
    for (int i = 0; i < n; ++i) {
        const interp_compress_item &it = items[i];
        const interp_config &c = it.cfg;
        const Dims d = to_dims(it.dims);
        unsigned char *ws = static_cast<unsigned char *>(it.d_ws);
        uint32_t *bitmap = reinterpret_cast<uint32_t *>(ws + L[i].bitmap);
        uint32_t *blockcnt = reinterpret_cast<uint32_t *>(ws + L[i].blockcnt);
        pro[i] = prologue_item(it, L[i]);
        if (is_nd(c.ndim))
            args[i] = gi::CompressArgs{it.d_x, d, it.d_anchors, it.d_codes, bitmap, blockcnt, it.d_hist, c.radius,
                                       it.d_hdr, false, false, 1};
        else
            args3[n3++] = args[i] =
                gi::CompressArgs{it.d_x, d, it.d_anchors, it.d_codes, bitmap, blockcnt, it.d_hist, c.radius,
                                 it.d_hdr, gi::aligned16(it.d_codes) && d.nx % 8 == 0, c.domain_x == 32,
                                 code_store_width(it.d_codes, d.nx)};
    }
    cudaError_t e = gi::launch_prologue(pro, n, s);
    if (e == cudaSuccess) {
        timing_mark(0, 0, s);
        const gi::TileSchedule ts{sched ? sched->run : 0, sched ? sched->ctas_per_sm : 0};
        if (n3 > 0) e = gi::launch_compress_tiles(args3, n3, s, &ts);  // one persistent launch for every 3-D field
        for (int i = 0; i < n && e == cudaSuccess; ++i)                // one launch per 1-D / 2-D field
            if (is_nd(items[i].cfg.ndim)) e = gi::launch_nd_compress(items[i].cfg.ndim, args[i], s);
        timing_mark(0, 1, s);
    }
    if (e == cudaSuccess) {
        // ordered compaction of every field in two launches; the 3-D tile kernel leaves bin R
        // to the scan, the 1-D / 2-D kernels count every bin and write row-major bitmaps
        gi::CompactItem ci[gi::kMaxBatch];
        for (int i = 0; i < n; ++i) {
            const interp_compress_item &it = items[i];
            const bool nd = is_nd(it.cfg.ndim);
            ci[i] = gi::CompactItem{args[i].bitmap, args[i].blockcnt, L[i].words, args[i].dims, it.d_x,
                                    it.d_out_idx, it.d_out_val, it.out_capacity, it.d_hdr, nd,
                                    nd ? nullptr : it.d_hist, it.cfg.radius};
        }
        e = gi::launch_outlier_compaction(ci, n, s);
    }
    return cuda_status(e);
}

int interp_compress(const float *d_x, const int64_t dims[3], double eb, const interp_config *cfg,
                    float *d_anchors, uint16_t *d_codes, uint32_t *d_out_idx, float *d_out_val,
                    uint64_t out_capacity, uint32_t *d_hist, interp_header *d_hdr, void *d_ws, size_t ws_bytes,
                    interp_stream_t stream)
{
    if (!dims_ok(dims) || !cfg) return INTERP_EINVAL;
    interp_compress_item it;
    it.d_x = d_x;
    for (int a = 0; a < 3; ++a) it.dims[a] = dims[a];
    it.eb = eb;
    it.cfg = *cfg;
    it.d_anchors = d_anchors;
    it.d_codes = d_codes;
    it.d_out_idx = d_out_idx;
    it.d_out_val = d_out_val;
    it.out_capacity = out_capacity;
    it.d_hist = d_hist;
    it.d_hdr = d_hdr;
    it.d_ws = d_ws;
    it.ws_bytes = ws_bytes;
    if (cfg->ndim == 1 || cfg->ndim == 2) return compress_nd(it, stream);
    return interp_compress_batched(&it, 1, stream);
}

int interp_decompress_batched(const interp_decompress_item *items, int n, interp_stream_t stream)
{
    return interp_decompress_batched_scheduled(items, n, nullptr, stream);
}

int interp_decompress_batched_scheduled(const interp_decompress_item *items, int n,
                                        const interp_tile_schedule *sched, interp_stream_t stream)
{
    if (sched && (sched->run < 0 || sched->ctas_per_sm < 0)) return INTERP_EINVAL;
    if (!items || n < 1 || n > gi::kMaxBatch) return INTERP_EINVAL;
    for (int i = 0; i < n; ++i) {
        const interp_decompress_item &it = items[i];
        if (!dims_ok(it.dims) || it.ndim < 0 || it.ndim > 3) return INTERP_EINVAL;
        if (!it.d_hdr || !it.d_anchors || !it.d_codes || !it.d_xrec) return INTERP_EINVAL;
        if (it.out_capacity > 0 && (!it.d_out_idx || !it.d_out_val)) return INTERP_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    gi::DecompressArgs args[gi::kMaxBatch], args3[gi::kMaxBatch];
    gi::ScatterItem sc[gi::kMaxBatch];
    int nsc = 0, n3 = 0;
    for (int i = 0; i < n; ++i) {
        const interp_decompress_item &it = items[i];
        const Dims d = to_dims(it.dims);
        if (it.out_capacity > 0) sc[nsc++] = gi::ScatterItem{it.d_hdr, it.d_out_idx, it.d_out_val, it.out_capacity,
                                                             it.d_xrec};
        if (is_nd(it.ndim))
            args[i] = gi::DecompressArgs{d, it.d_anchors, it.d_codes, it.d_xrec, it.d_hdr, false};
        else
            args3[n3++] = args[i] = gi::DecompressArgs{d, it.d_anchors, it.d_codes, it.d_xrec, it.d_hdr,
                                                       gi::aligned16(it.d_xrec) && d.nx % 4 == 0, it.d_out_idx,
                                                       it.out_capacity};
    }
    // every field's stored outlier values in one launch, then one tile launch for the 3-D
    // fields and one per 1-D / 2-D field
    cudaError_t e = nsc > 0 ? gi::launch_outlier_scatter(sc, nsc, s) : cudaSuccess;
    if (e == cudaSuccess) {
        timing_mark(1, 0, s);
        const gi::TileSchedule ts{sched ? sched->run : 0, sched ? sched->ctas_per_sm : 0};
        if (n3 > 0) e = gi::launch_decompress_tiles(args3, n3, s, &ts);
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            if (is_nd(items[i].ndim)) e = gi::launch_nd_decompress(items[i].ndim, args[i], s);
        timing_mark(1, 1, s);
    }
    return cuda_status(e);
}

int interp_decompress(const int64_t dims[3], const interp_header *d_hdr, const float *d_anchors,
                      const uint16_t *d_codes, const uint32_t *d_out_idx, const float *d_out_val,
                      uint64_t out_capacity, float *d_xrec, interp_stream_t stream)
{
    if (!dims_ok(dims)) return INTERP_EINVAL;
    interp_decompress_item it;
    for (int a = 0; a < 3; ++a) it.dims[a] = dims[a];
    it.d_hdr = d_hdr;
    it.d_anchors = d_anchors;
    it.d_codes = d_codes;
    it.d_out_idx = d_out_idx;
    it.d_out_val = d_out_val;
    it.out_capacity = out_capacity;
    it.d_xrec = d_xrec;
    it.ndim = 3;
    return interp_decompress_batched(&it, 1, stream);
}

int interp_decompress_nd(int32_t ndim, const int64_t dims[3], const interp_header *d_hdr,
                         const float *d_anchors, const uint16_t *d_codes, const uint32_t *d_out_idx,
                         const float *d_out_val, uint64_t out_capacity, float *d_xrec, interp_stream_t stream)
{
    if (ndim == 0 || ndim == 3)
        return interp_decompress(dims, d_hdr, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_xrec,
                                 stream);
    if (ndim != 1 && ndim != 2) return INTERP_EINVAL;
    if (!dims_ok(dims)) return INTERP_EINVAL;
    if (!d_hdr || !d_anchors || !d_codes || !d_xrec) return INTERP_EINVAL;
    if (out_capacity > 0 && (!d_out_idx || !d_out_val)) return INTERP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Dims d = to_dims(dims);
    cudaError_t e = cudaSuccess;
    if (out_capacity > 0) {
        const gi::ScatterItem sc{d_hdr, d_out_idx, d_out_val, out_capacity, d_xrec};
        e = gi::launch_outlier_scatter(&sc, 1, s);
    }
    const gi::DecompressArgs args{d, d_anchors, d_codes, d_xrec, d_hdr, false};
    if (e == cudaSuccess) {
        timing_mark(1, 0, s);
        e = gi::launch_nd_decompress(ndim, args, s);
        timing_mark(1, 1, s);
    }
    return cuda_status(e);
}

int qcode_histogram(const uint16_t *d_codes, uint64_t n, int32_t radius, uint32_t *d_hist, interp_stream_t stream)
{
    if (radius < 2 || radius > 32768 || !d_hist || (n > 0 && !d_codes)) return INTERP_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * 2 * (size_t)radius, s);
    if (e == cudaSuccess && n > 0) e = gi::launch_histogram(d_codes, n, radius, d_hist, s);
    return cuda_status(e);
}

size_t interp_quality_workspace_bytes(void) { return gi::quality_workspace_bytes(); }

int interp_quality_report(const uint32_t *d_hist, int32_t radius, const float *d_x, const float *d_xrec, uint64_t n,
                          interp_quality *d_out, void *d_ws, size_t ws_bytes, interp_stream_t stream)
{
    if (radius < 2 || radius > 32768 || !d_hist || !d_out) return INTERP_EINVAL;
    if ((d_x == nullptr) != (d_xrec == nullptr)) return INTERP_EINVAL;
    if (d_x && (!d_ws || ws_bytes < gi::quality_workspace_bytes())) return INTERP_EWORKSPACE;
    return cuda_status(gi::launch_quality(d_hist, radius, d_x, d_xrec, n, d_out, d_ws,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

int interp_huffman_codebook(const uint32_t *h_hist, int32_t radius, int32_t max_len, uint8_t *h_lengths,
                            uint32_t *h_codewords)
{
    if (radius < 2 || radius > 32768 || !h_hist || !h_lengths || !h_codewords) return INTERP_EINVAL;
    if (max_len < 1 || max_len > gi::huffman_max_len()) return INTERP_EINVAL;
    return gi::huffman_codebook(h_hist, 2 * radius, max_len, h_lengths, h_codewords) ? INTERP_OK : INTERP_EINVAL;
}

uint64_t interp_huffman_chunks(uint64_t n) { return gi::huffman_chunks(n); }

uint64_t interp_huffman_capacity_words(uint64_t n, int32_t max_len)
{
    if (max_len < 1 || max_len > gi::huffman_max_len()) return 0;
    return gi::huffman_capacity_words(n, max_len);
}

size_t interp_huffman_workspace_bytes(uint64_t n, int32_t radius)
{
    if (radius < 2 || radius > 32768 || n >= (1ull << 32)) return 0;
    return 256 + std::max(gi::huffman_decode_workspace(2 * radius), gi::huffman_encode_workspace(n));
}

int interp_huffman_encode(const uint16_t *d_codes, uint64_t n, int32_t radius, const uint8_t *d_lengths,
                          const uint32_t *d_codewords, uint32_t *d_offsets, uint32_t *d_words,
                          uint64_t capacity_words, void *d_ws, size_t ws_bytes, interp_stream_t stream)
{
    if (radius < 2 || radius > 32768 || !d_lengths || !d_codewords || !d_offsets || !d_ws) return INTERP_EINVAL;
    if (n > 0 && (!d_codes || !d_words)) return INTERP_EINVAL;
    if (n >= (1ull << 32)) return INTERP_EINVAL;
    if (ws_bytes < interp_huffman_workspace_bytes(n, radius)) return INTERP_EWORKSPACE;
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    unsigned int *bad = reinterpret_cast<unsigned int *>(ws);
    return cuda_status(gi::launch_huffman_encode(d_codes, n, d_lengths, d_codewords, 2 * radius, d_offsets, d_words,
                                                 capacity_words, reinterpret_cast<uint32_t *>(ws + 256), bad,
                                                 reinterpret_cast<cudaStream_t>(stream)));
}

int interp_huffman_decode(const uint32_t *d_words, const uint32_t *d_offsets, uint64_t n, int32_t radius,
                          const uint8_t *d_lengths, const uint32_t *d_codewords, uint16_t *d_codes, void *d_ws,
                          size_t ws_bytes, interp_stream_t stream)
{
    if (radius < 2 || radius > 32768 || !d_lengths || !d_codewords || !d_offsets || !d_ws) return INTERP_EINVAL;
    if (n > 0 && (!d_codes || !d_words)) return INTERP_EINVAL;
    if (n >= (1ull << 32)) return INTERP_EINVAL;
    if (ws_bytes < interp_huffman_workspace_bytes(n, radius)) return INTERP_EWORKSPACE;
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    unsigned int *bad = reinterpret_cast<unsigned int *>(ws);
    return cuda_status(gi::launch_huffman_decode(d_words, d_offsets, n, d_lengths, d_codewords, 2 * radius, d_codes,
                                                 ws + 256, bad, reinterpret_cast<cudaStream_t>(stream)));
}

double interp_alpha(double eps) { return alpha_of_eps(eps); }

int interp_value_range(const float *d_x, const int64_t dims[3], float *d_range, void *d_ws, size_t ws_bytes,
                       interp_stream_t stream)
{
    if (!dims_ok(dims) || !d_x || !d_range || !d_ws) return INTERP_EINVAL;
    if (ws_bytes < kCtrlBytes + gi::range_partials_bytes()) return INTERP_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    unsigned int *counter = reinterpret_cast<unsigned int *>(ws);
    cudaError_t e = cudaMemsetAsync(ws, 0, kCtrlBytes, s);
    if (e == cudaSuccess) {
        interp_config unused{};
        e = gi::launch_range(d_x, to_dims(dims), 0.0, unused, 1.0, nullptr, ws + kCtrlBytes, counter,
                             gi::range_blocks(), s, d_range);
    }
    return cuda_status(e);
}

int interp_autotune(const float *d_x, const int64_t dims[3], interp_config *h_cfg, double *h_profile, void *d_ws,
                    size_t ws_bytes, interp_stream_t stream)
{
    if (!dims_ok(dims) || !h_cfg || !d_x || !d_ws) return INTERP_EINVAL;
    if (ws_bytes < sizeof(interp_header)) return INTERP_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    interp_header *tmp = static_cast<interp_header *>(d_ws);
    if (h_cfg->ndim < 0 || h_cfg->ndim > 3) return INTERP_EINVAL;
    cudaError_t e = gi::launch_profile(d_x, to_dims(dims), tmp, 1, s, h_cfg->ndim);
    interp_header h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tmp, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return INTERP_ECUDA;
    for (int a = 0; a < 3; ++a) {
        h_cfg->dim_order[a] = h.cfg.dim_order[a];
        h_cfg->cubic_kind[a] = h.cfg.cubic_kind[a];
        h_cfg->level_kind[a] = h.cfg.level_kind[a];
    }
    if (h_profile) std::memcpy(h_profile, h.profile, sizeof(h.profile));
    return INTERP_OK;
}

int interp_timing_enable(int on)
{
    if (on && !g_timing.created) {
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < kTimingPairs; ++i)
                for (int j = 0; j < 2; ++j)
                    if (cudaEventCreate(&g_timing.ev[k][i][j]) != cudaSuccess) return INTERP_ECUDA;
        g_timing.created = true;
    }
    if (on) g_timing.used[0] = g_timing.used[1] = 0;
    g_timing.on = on != 0;
    return INTERP_OK;
}

int interp_timing_read(double *compress_ms, int32_t *compress_launches, double *decompress_ms,
                       int32_t *decompress_launches)
{
    double ms[2] = {0.0, 0.0};
    for (int k = 0; k < 2 && g_timing.created; ++k)
        for (int i = 0; i < g_timing.used[k]; ++i) {
            if (cudaEventSynchronize(g_timing.ev[k][i][1]) != cudaSuccess) return INTERP_ECUDA;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, g_timing.ev[k][i][0], g_timing.ev[k][i][1]) != cudaSuccess)
                return INTERP_ECUDA;
            ms[k] += t;
        }
    if (compress_ms) *compress_ms = ms[0];
    if (compress_launches) *compress_launches = g_timing.used[0];
    if (decompress_ms) *decompress_ms = ms[1];
    if (decompress_launches) *decompress_launches = g_timing.used[1];
    return INTERP_OK;
}

const char *interp_status_string(int status)
{
    switch (status) {
    case INTERP_OK: return "ok";
    case INTERP_EINVAL: return "invalid argument";
    case INTERP_ECUDA: return "CUDA error";
    case INTERP_EWORKSPACE: return "workspace too small";
    case INTERP_ECAPACITY: return "outlier capacity exceeded";
    case INTERP_ENONFINITE: return "non-finite input";
    case INTERP_ESCRATCH: return "field too large for the built-in no-allocation scratch";
    default: return "unknown status";
    }
}

}  // extern "C"
