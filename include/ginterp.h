/*
 * ginterp.h -- C ABI of the GB300 G-Interp library (libginterp.so).
 *
 * G-Interp is the interpolation predictor-quantizer of the cuSZ-i lossy
 * compressor (arXiv 2312.05492, Sec. IV): anchors on a stride-8 grid are
 * stored losslessly (Sec. IV-A); the remaining points are predicted level by
 * level at strides 4, 2, 1, one axis at a time, by linear / quadratic / cubic
 * splines chosen by neighbour count (Sec. IV-B.1, Fig. 3) from already
 * reconstructed values; each residual is quantized against a level-wise error
 * bound (Sec. IV-B.1) into a 16-bit quant-code, codes too large for the
 * radius R become outliers (Sec. III-A) gathered by stream compaction
 * (Sec. V-A), and the codes are histogrammed (Fig. 1, Sec. V-A).
 * Decompression replays the same order (Sec. IV-B.1).
 *
 * Conventions for every entry point:
 *   - Fields are float32, C-contiguous, dims = {nz, ny, nx} with x fastest:
 *     index i = (z*ny + y)*nx + x.  1 <= each dim, N = nz*ny*nx < 2^32.
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *     are host pointers.  The caller allocates and owns every buffer; the
 *     library never allocates, frees or synchronises (except interp_autotune).
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is stream-ordered.  Input buffers are not modified.
 *   - Return value: INTERP_OK, or a negative interp_status for argument
 *     errors (detected on the host before anything is enqueued) and launch
 *     errors.  Conditions found on the device are reported in
 *     interp_header.status (bit flags INTERP_STATUS_*).
 *   - Level index l = 0, 1, 2, ... refers to strides 1, 2, 4, ... (the paper's
 *     level ell = l + 1); per-level arrays are indexed by l.  The header keeps
 *     the bounds of l = 0..2; the 1-D and 2-D geometries (cfg.ndim) continue
 *     e_l = e / alpha^l to their 9 and 4 levels.
 */
#ifndef GINTERP_H
#define GINTERP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *interp_stream_t; /* identical to cudaStream_t */

typedef enum {
    INTERP_OK = 0,
    INTERP_EINVAL = -1,     /* bad argument (dims, eb, radius, order, null pointer, ...) */
    INTERP_ECUDA = -2,      /* a CUDA launch or runtime call failed */
    INTERP_EWORKSPACE = -3, /* workspace smaller than interp_workspace_bytes() */
    INTERP_ECAPACITY = -4,  /* (host helper) outlier count exceeds out_capacity */
    INTERP_ENONFINITE = -5, /* (host helper) non-finite input values were found */
    INTERP_ESCRATCH = -6    /* interp_compress_noalloc: the field needs more scratch than the
                               library's built-in array (interp_noalloc_scratch_bytes()) */
} interp_status;

/* device-side status bits (interp_header.status) */
#define INTERP_STATUS_CAPACITY 1u  /* more outliers than out_capacity; n_outliers is the true count */
#define INTERP_STATUS_NONFINITE 2u /* the field holds NaN/Inf (stored losslessly as outliers) */
#define INTERP_STATUS_TIMEOUT 4u   /* a tile kernel gave up waiting for an input transfer;
                                      set by compression and decompression.  The call's outputs
                                      are then invalid, and a transfer that never completed
                                      points to a device fault: stop using the CUDA context
                                      (the kernel waits once more, bounded, before it exits) */

/* Interpolation configuration (Sec. IV-B). */
typedef struct {
    int32_t dim_order[3];  /* permutation of {0=z, 1=y, 2=x}; dim_order[0] is interpolated
                              first in every level (Sec. IV-B.2: least smooth axis first) */
    int32_t level_kind[3]; /* per level l (stride 2^l): 0 = linear spline only,
                              1 = splines by neighbour count (cubic/quadratic/linear) */
    int32_t cubic_kind[3]; /* per axis: 0 = not-a-knot cubic, 1 = natural cubic */
    int32_t eb_mode;       /* 0 = eb is absolute, 1 = eb is relative to the value range */
    int32_t autotune;      /* 1 = dim_order, cubic_kind and level_kind are chosen on the
                              device from a 4x4x4 sampling profile (Sec. IV-B.2) */
    int32_t radius;        /* R: codes q with |q| < R are kept, others become outliers;
                              2 <= R <= 32768 (codes are uint16, code 0 marks an outlier) */
    int32_t domain_x;      /* neighbour domain along x: 0 or 8 = the closed 8^3 chunk
                              (Sec. IV-A, Fig. 3); 32 = the closed 32-point block of the
                              32x8x8 data blocks, whose four chunks share points along x
                              (Sec. IV-C).  Anchors stay on the stride-8 grid either way. */
    int32_t ndim;          /* chunk geometry (Sec. IV-A): 0 or 3 = 8^3 chunks, strides 4, 2, 1;
                              2 = 16^2 chunks over (y, x), strides 8 .. 1, every z-slice on its
                              own; 1 = 512-point chunks along x, strides 256 .. 1, every (z, y)
                              row on its own.  Levels coarser than stride 4 use level_kind[2];
                              their bounds continue e_l = e / alpha^l.  1 and 2 need domain_x
                              0 or 8 and are taken by interp_compress / interp_decompress_nd,
                              the batched forms and the no-allocation form. */
    double alpha;          /* error-bound reduction factor; <= 0 selects Eq. 1 A(eps) in
                              relative mode and 1 in absolute mode */
} interp_config;

/* Written on the device by interp_compress; read by interp_decompress. */
typedef struct {
    int64_t dims[3];
    interp_config cfg;     /* effective configuration (after autotuning) */
    double eb;             /* eb as passed by the caller */
    double eb_abs;         /* absolute bound e = eps * (vmax - vmin) or eb */
    double alpha;          /* effective alpha */
    float e[3];            /* level bounds e_l = e / alpha^l (Sec. IV-B.1) */
    float twoe[3];         /* 2 e_l: quantization bin width */
    float inv2e[3];        /* float(1 / (2 e_l)) */
    float vmin, vmax;      /* finite value range (relative mode) */
    uint64_t n_outliers;   /* true number of outliers */
    uint64_t n_nonfinite;  /* non-finite input values (relative mode) */
    uint32_t status;       /* INTERP_STATUS_* bits */
    uint32_t reserved;
    double profile[18];    /* sampling-profile error sums (autotune) */
} interp_header;

/* Number of anchor points: prod over axes of (floor((n_d - 1) / 8) + 1) (Sec. IV-A).
 * Returns 0 for invalid dims. */
size_t interp_anchor_count(const int64_t dims[3]);

/* Anchor count of the ndim-D geometry (cfg.ndim): prod over axes of
 * (floor((n_d - 1) / A_d) + 1) with A_d the chunk edge (8, 16 or 512) on the last
 * ndim axes and 1 on the others.  0 for invalid dims or ndim. */
size_t interp_anchor_count_nd(const int64_t dims[3], int32_t ndim);

/* Device scratch that interp_compress needs, in bytes (0 for invalid args). */
size_t interp_workspace_bytes(const int64_t dims[3], const interp_config *cfg);

/* Compress a float32 field (Sec. IV-A/B, Sec. V-A).
 *   d_x          [N] input field (read only)
 *   dims         host array {nz, ny, nx}
 *   eb           error bound: absolute, or relative to (max - min) when cfg->eb_mode = 1
 *   cfg          host pointer to the configuration (copied; not retained)
 *   d_anchors    [interp_anchor_count(dims)] out: x at points with all coords = 0 mod 8,
 *                laid out [nz'][ny'][nx'] with n' = floor((n - 1)/8) + 1 (for cfg->ndim
 *                1 or 2: [interp_anchor_count_nd(dims, ndim)], the chunked coords = 0
 *                mod 512 / 16, every index along the other axes)
 *   d_codes      [N] out: uint16 quant-codes; q + R for kept points, 0 for outliers,
 *                R at anchors
 *   d_out_idx,
 *   d_out_val    [out_capacity] out: outlier indices (ascending) and original values;
 *                if the true count exceeds out_capacity only the first out_capacity
 *                are written and INTERP_STATUS_CAPACITY is set
 *   d_hist       [2R] out or NULL: histogram of d_codes (zeroed by the callee)
 *   d_hdr        out: device header (bounds, effective config, counts, status)
 *   d_ws         device scratch of ws_bytes >= interp_workspace_bytes(dims, cfg)
 * Guarantee: for every point |x - x'| <= e_l of its level, where x' is the output of
 * interp_decompress and e_l = float(eb_abs / alpha^l) (header e[l] for l <= 2); e_0, the
 * largest, is eb_abs rounded to float, so it may exceed eb_abs by up to half a float ulp.
 * Anchors and outliers are exact.  Fields compressed with cfg->ndim 1 or 2 are
 * decompressed by interp_decompress_nd. */
int interp_compress(const float *d_x, const int64_t dims[3], double eb, const interp_config *cfg,
                    float *d_anchors, uint16_t *d_codes, uint32_t *d_out_idx, float *d_out_val,
                    uint64_t out_capacity, uint32_t *d_hist, interp_header *d_hdr,
                    void *d_ws, size_t ws_bytes, interp_stream_t stream);

/* Decompress (Sec. IV-B.1: replay of the prediction from the quant-codes).
 *   dims must equal the dims the field was compressed with (the caller keeps
 *   them; they are also in the header); d_hdr, d_anchors, d_codes, d_out_idx,
 *   d_out_val as written by interp_compress, with out_capacity entries
 *   available (the first min(n_outliers, out_capacity) are scattered);
 *   d_xrec [N] out.  No workspace is needed. */
int interp_decompress(const int64_t dims[3], const interp_header *d_hdr, const float *d_anchors,
                      const uint16_t *d_codes, const uint32_t *d_out_idx, const float *d_out_val,
                      uint64_t out_capacity, float *d_xrec, interp_stream_t stream);

/* interp_decompress for a field compressed with cfg.ndim = ndim (1, 2 or 3; 3 is
 * interp_decompress itself).  Same arguments and results. */
int interp_decompress_nd(int32_t ndim, const int64_t dims[3], const interp_header *d_hdr,
                         const float *d_anchors, const uint16_t *d_codes, const uint32_t *d_out_idx,
                         const float *d_out_val, uint64_t out_capacity, float *d_xrec, interp_stream_t stream);

/* Batched forms: n fields of any (uneven) shapes, bounds and configurations in one call.
 * Each item carries exactly the arguments of the single-field call (its own workspace).
 * The set-up of all fields (workspace clear; range, profile, bounds), their outlier
 * compaction and, for decompression, their outlier scatter take one launch per phase for
 * the whole batch.  The tile work of all 3-D fields runs in ONE persistent kernel launch
 * whose CTAs take work items (runs of 8-plane slabs of 16 x 32 columns) from all of them;
 * 1-D / 2-D fields (interp_config.ndim 1 or 2 when compressing, the item's ndim when
 * decompressing) take one tile launch each.  Results are identical, bit for bit, to n
 * single calls.  1 <= n <= 16.  Stream-ordered, no synchronisation; capturable into a CUDA
 * graph after one warm-up call on the device. */
typedef struct {
    const float *d_x;
    int64_t dims[3];
    double eb;
    interp_config cfg;
    float *d_anchors;
    uint16_t *d_codes;
    uint32_t *d_out_idx;
    float *d_out_val;
    uint64_t out_capacity;
    uint32_t *d_hist;
    interp_header *d_hdr;
    void *d_ws;
    size_t ws_bytes;
} interp_compress_item;

typedef struct {
    int64_t dims[3];
    const interp_header *d_hdr;
    const float *d_anchors;
    const uint16_t *d_codes;
    const uint32_t *d_out_idx;
    const float *d_out_val;
    uint64_t out_capacity;
    float *d_xrec;
    int32_t ndim; /* the field's chunk geometry, its interp_config.ndim at compression:
                     0 or 3 = 3-D, 1 / 2 = 1-D / 2-D chunks (interp_decompress_nd); others
                     INTERP_EINVAL */
} interp_decompress_item;

int interp_compress_batched(const interp_compress_item *h_items, int n, interp_stream_t stream);
int interp_decompress_batched(const interp_decompress_item *h_items, int n, interp_stream_t stream);

/* Schedule of the persistent tile launch of a (batched) call.  The paper has no
 * counterpart: it is a launch parameter of this library's GPU mapping.  run = slabs of 8
 * planes per work item (0 = the library's cost model; larger runs recompute fewer
 * closing planes, shorter ones balance the CTAs better), ctas_per_sm = resident CTAs
 * per SM (0 = the occupancy limit; a smaller value caps it).  Outputs do not depend on
 * the schedule, bit for bit. */
typedef struct {
    int32_t run;
    int32_t ctas_per_sm;
} interp_tile_schedule;

/* interp_compress_batched / interp_decompress_batched with an explicit schedule
 * (h_sched may be NULL: automatic).  Negative fields are INTERP_EINVAL. */
int interp_compress_batched_scheduled(const interp_compress_item *h_items, int n, const interp_tile_schedule *h_sched,
                                      interp_stream_t stream);
int interp_decompress_batched_scheduled(const interp_decompress_item *h_items, int n,
                                        const interp_tile_schedule *h_sched, interp_stream_t stream);

/* Tile-schedule autotuner of a batch: runs the batch's compression (h_citems) and then
 * its decompression (h_ditems, which must read what h_citems write) with every
 * candidate schedule (runs 1, 2, 4, 8, 16, whole columns and the cost model's choice;
 * the occupancy limit and one or two CTAs per SM fewer), times each on `stream` with
 * CUDA events (one warm-up call, then the mean of two) and returns the fastest in
 * h_csched / h_dsched.  The outputs are written and valid afterwards.  Synchronises
 * `stream`.  Results are cached by the fields' shapes, configurations, bounds and
 * buffer alignment: a later call with the same batch returns the cached schedules
 * without running anything unless force != 0. */
int interp_tune_batched(const interp_compress_item *h_citems, const interp_decompress_item *h_ditems, int n,
                        int32_t force, interp_tile_schedule *h_csched, interp_tile_schedule *h_dsched,
                        interp_stream_t stream);

/* Histogram of quant-codes (Fig. 1 "histogram", Sec. V-A): d_hist[c] = #{i : codes[i] = c}
 * for c in [0, 2R); d_hist (2R uint32) is zeroed by the callee.  Codes >= 2R are ignored. */
int qcode_histogram(const uint16_t *d_codes, uint64_t n, int32_t radius, uint32_t *d_hist,
                    interp_stream_t stream);

/* Eq. 1 (Sec. IV-B.2): the level-bound reduction factor alpha = A(eps) for a relative
 * bound eps, the value interp_compress uses in relative mode when cfg->alpha <= 0
 * (piecewise linear between 1 at eps <= 1e-5 and 2 at eps >= 1e-1).  Host-only, pure. */
double interp_alpha(double eps);

/* Value range of a field (Sec. IV-B.1: a relative bound is scaled by the value range):
 * writes {vmin, vmax} over the finite values of d_x (N = dims product floats,
 * contiguous) to d_range (2 floats, device); {0, 0} when no value is finite.  This is
 * the reduction interp_compress runs in relative mode; a caller that splits one field
 * across GPUs reduces the per-part ranges and passes eps * (vmax - vmin) as an absolute
 * bound.  d_ws: any workspace sized by interp_workspace_bytes() for the same dims.
 * Stream-ordered, no synchronisation; errors as interp_compress. */
int interp_value_range(const float *d_x, const int64_t dims[3], float *d_range, void *d_ws, size_t ws_bytes,
                       interp_stream_t stream);

/* Sampling profile and decision (Sec. IV-B.1 data profiling, Sec. IV-B.2 auto-tuning):
 * fills h_cfg->dim_order, cubic_kind and level_kind from the 4x4x4 sample profile of
 * d_x (along the chunked axes of h_cfg->ndim only; the other axes' sums are 0 and they
 * sort last) and writes the 18 profile sums to h_profile (may be NULL).  Uses 512 bytes of
 * d_ws.  SYNCHRONISES the stream (one small device-to-host copy). */
int interp_autotune(const float *d_x, const int64_t dims[3], interp_config *h_cfg,
                    double *h_profile, void *d_ws, size_t ws_bytes, interp_stream_t stream);

/* Quality report of a compression (Sec. IV-D: Fig. 4 counts nonzero quant-codes; the
 * PSNR comparison after it).  From the code histogram (2R bins, as written by
 * interp_compress or qcode_histogram): the point count, outliers, nonzero quant-codes,
 * the largest |q| among kept points and the Shannon entropy of the codes in bits per
 * point (the rate an entropy coder approaches: 32 / entropy_bits estimates the ratio of
 * the code stream).  From the field and its reconstruction (optional, both or neither):
 * the sum and maximum of the error over finite points, the finite value range and the
 * PSNR.  Not part of the compression path. */
typedef struct {
    uint64_t n;           /* points in the histogram */
    uint64_t n_outliers;  /* code 0 */
    uint64_t n_nonzero;   /* points whose quant-code is not 0 (code != R), outliers included */
    uint64_t n_finite;    /* finite points of x in the error statistics (0 without x) */
    int32_t max_abs_q;    /* largest |code - R| among kept points (code != 0) */
    int32_t reserved;
    double entropy_bits;  /* -sum_c p_c log2 p_c, p_c = hist[c] / n */
    double sse;           /* sum of (x - x')^2 over finite x, in double (NaN without x) */
    double max_abs_err;   /* max |x - x'| over finite x */
    double vmin, vmax;    /* finite value range of x */
    double psnr_db;       /* 20 log10(vmax - vmin) - 10 log10(sse / n_finite); +Inf if sse = 0 */
} interp_quality;

/* Scratch interp_quality_report needs (bytes). */
size_t interp_quality_workspace_bytes(void);

/* Fill *d_out (device) from d_hist (2R uint32) and, when both are non-NULL, from
 * d_x and d_xrec (N floats each).  Stream-ordered; d_ws holds at least
 * interp_quality_workspace_bytes() bytes.  The error sums are accumulated in double
 * in a fixed order for a given device, so they match a float64 sum to rounding. */
int interp_quality_report(const uint32_t *d_hist, int32_t radius, const float *d_x, const float *d_xrec,
                          uint64_t n, interp_quality *d_out, void *d_ws, size_t ws_bytes, interp_stream_t stream);

/* ---- Canonical Huffman coding of the quant-codes (Sec. V-A: the lossless stage after
 * the histogram; the codebook is built on the host, the codes are encoded and decoded on
 * the GPU).  Stream: the codes are cut into chunks of 1024; a chunk's codewords are
 * concatenated most-significant bit first into 32-bit words (its first bit is bit 31 of
 * its first word) and padded with zero bits to a whole word; d_offsets[k] is chunk k's
 * first word and d_offsets[nchunks] the total number of words. */

/* Host only.  Code lengths and canonical codewords for the 2R symbols of h_hist (uint32
 * counts): Huffman's construction (the two lightest subtrees merge first; ties by weight,
 * then creation order: symbols by index, merged subtrees after), then, if a length
 * exceeds max_len (1..24), lengths above it are cut to max_len, then, while the Kraft
 * sum exceeds 1, the codeword that is longest among those shorter than max_len gains one
 * bit (on equal lengths the lighter symbol, on equal counts the higher index); canonical
 * codewords assign consecutive values in (length, symbol) order.  Unused symbols get
 * length 0; a single used symbol gets length 1.  h_lengths [2R] and h_codewords [2R] are
 * outputs.  INTERP_EINVAL when more than 2^max_len symbols are used (no prefix code of
 * max_len bits holds them). */
int interp_huffman_codebook(const uint32_t *h_hist, int32_t radius, int32_t max_len, uint8_t *h_lengths,
                            uint32_t *h_codewords);

/* Number of 1024-code chunks for n codes, and the words of stream room that always
 * suffice with codewords of at most max_len bits. */
uint64_t interp_huffman_chunks(uint64_t n);
uint64_t interp_huffman_capacity_words(uint64_t n, int32_t max_len);

/* Scratch for interp_huffman_encode / interp_huffman_decode of n codes (bytes; 0 for
 * a radius outside 2..32768 or n >= 2^32). */
size_t interp_huffman_workspace_bytes(uint64_t n, int32_t radius);

/* Encode n codes (each < 2R, every one with a nonzero length in d_lengths) with the
 * codebook (d_lengths [2R], d_codewords [2R], device copies of interp_huffman_codebook's
 * output).  Writes d_offsets [chunks + 1] and the stream d_words (capacity_words words,
 * at least the used d_offsets[chunks]).  A chunk that would not fit, or a codebook with
 * longer codewords than 24 bits, sets the device flag at the start of d_ws to 1 (0 on
 * success); nothing outside d_words' capacity is written.  Stream-ordered. */
int interp_huffman_encode(const uint16_t *d_codes, uint64_t n, int32_t radius, const uint8_t *d_lengths,
                          const uint32_t *d_codewords, uint32_t *d_offsets, uint32_t *d_words,
                          uint64_t capacity_words, void *d_ws, size_t ws_bytes, interp_stream_t stream);

/* Decode the stream back into n codes (d_codes [n]) with the same codebook.  A word
 * sequence that is not a codeword sets the device flag at the start of d_ws to 1.
 * Stream-ordered. */
int interp_huffman_decode(const uint32_t *d_words, const uint32_t *d_offsets, uint64_t n, int32_t radius,
                          const uint8_t *d_lengths, const uint32_t *d_codewords, uint16_t *d_codes, void *d_ws,
                          size_t ws_bytes, interp_stream_t stream);

/* Measurement support (not part of the compression method): while enabled,
 * every interp_compress / interp_decompress call records a pair of CUDA events
 * on its stream immediately around its tile kernel (at most 512 pairs per kernel;
 * later calls are not recorded).  interp_timing_enable(1) clears previous
 * records, (0) stops recording.  interp_timing_read waits for the recorded
 * events and returns the summed milliseconds and launch counts of the
 * compression and decompression tile kernels (any pointer may be NULL).
 * Process-wide state for the current device; not thread-safe. */
int interp_timing_enable(int on);
int interp_timing_read(double *compress_ms, int32_t *compress_launches, double *decompress_ms,
                       int32_t *decompress_launches);

/* Compression without any caller-provided scratch (no counterpart in the paper).
 * For callers that cannot allocate device memory: their device memory belongs to an
 * allocator they cannot ask for more, they run in a host that forbids device allocation,
 * or they must never pay for a cudaMalloc and its synchronisation.  Same arguments and
 * results as interp_compress without d_ws / ws_bytes: the scratch is an array compiled
 * into the library (interp_noalloc_scratch_bytes() bytes, 24 MiB, held on every GPU that
 * loads the library until the process exits).  Fields whose interp_workspace_bytes()
 * exceed it are rejected with INTERP_ESCRATCH before any work is enqueued.  Every call
 * made outside stream capture looks up the array's device address on the current device
 * (so a device reset, which may move the array, is harmless); a call during capture uses
 * the address an earlier call on that device looked up, so make one call on the device
 * before capturing (INTERP_ECUDA otherwise).  Every call reuses the same array and clears
 * what must start at zero itself; calls whose work overlaps on the GPU race on it.  Not
 * thread-safe.  Allocates and frees nothing. */
int interp_compress_noalloc(const float *d_x, const int64_t dims[3], double eb, const interp_config *cfg,
                            float *d_anchors, uint16_t *d_codes, uint32_t *d_out_idx, float *d_out_val,
                            uint64_t out_capacity, uint32_t *d_hist, interp_header *d_hdr,
                            interp_stream_t stream);

/* Size in bytes of the built-in scratch array used by interp_compress_noalloc. */
size_t interp_noalloc_scratch_bytes(void);

/* Human-readable text for an interp_status value. */
const char *interp_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GINTERP_H */
