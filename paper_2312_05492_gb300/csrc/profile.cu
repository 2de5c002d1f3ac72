// Data profiling and auto-tuning (Sec. IV-B of arXiv 2312.05492):
//   - value range of the field -> absolute bound e = eps * (max - min)
//     and the level bounds e_l = e / alpha^l (Sec. IV-B.1), written to the
//     device header by the last CTA of the range reduction;
//   - the 4x4x4 sampling profile (two cubic splines per axis, Sec. IV-B.1)
//     and the configuration decision (Sec. IV-B.2), in one small CTA.
#include <algorithm>
#include <cfloat>
#include <cstring>

#include "common.cuh"

namespace gi {
namespace {

struct RangePartial {
    float lo, hi;
    unsigned long long nonfinite;
};

constexpr int RANGE_THREADS = 512;
constexpr int RANGE_MAX_BLOCKS = 4096;

// Header fields that depend only on the bound (Sec. IV-B.1): e_l = e / alpha^l,
// with alpha^l formed by multiplication in double.
__device__ void write_bounds(interp_header *h, Dims d, double eb, const interp_config &cfg, double alpha,
                             float vmin, float vmax, unsigned long long nonfinite)
{
    h->dims[0] = d.nz;
    h->dims[1] = d.ny;
    h->dims[2] = d.nx;
    if (!cfg.autotune) {
        for (int a = 0; a < 3; ++a) {
            h->cfg.dim_order[a] = cfg.dim_order[a];
            h->cfg.level_kind[a] = cfg.level_kind[a];
            h->cfg.cubic_kind[a] = cfg.cubic_kind[a];
        }
    }
    h->cfg.eb_mode = cfg.eb_mode;
    h->cfg.autotune = cfg.autotune;
    h->cfg.radius = cfg.radius;
    h->cfg.domain_x = cfg.domain_x;
    h->cfg.ndim = cfg.ndim;
    h->cfg.alpha = cfg.alpha;
    const double eb_abs = cfg.eb_mode ? eb * ((double)vmax - (double)vmin) : eb;
    h->eb = eb;
    h->eb_abs = eb_abs;
    h->alpha = alpha;
    double apow[3];
    apow[0] = 1.0;
    apow[1] = alpha;
    apow[2] = alpha * alpha;
    for (int l = 0; l < 3; ++l) {
        const float e = (float)(eb_abs / apow[l]);
        h->e[l] = e;
        h->twoe[l] = 2.0f * e;
        h->inv2e[l] = (float)(1.0 / (2.0 * (double)e));
    }
    h->vmin = vmin;
    h->vmax = vmax;
    h->n_outliers = 0;
    h->n_nonfinite = nonfinite;
    h->status = nonfinite ? INTERP_STATUS_NONFINITE : 0u;
    h->reserved = 0;
}

__global__ void k_header_init(interp_header *hdr, Dims d, double eb, interp_config cfg, double alpha)
{
    if (threadIdx.x == 0) write_bounds(hdr, d, eb, cfg, alpha, 0.0f, 0.0f, 0ull);
}

__device__ __forceinline__ void range_acc(float v, float &lo, float &hi, unsigned long long &bad)
{
    if (fabsf(v) <= FLT_MAX) {
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    } else {
        ++bad;
    }
}

// Block b of the nb blocks that reduce one field: grid-stride min/max over
// finite values with 4 independent 16-byte loads in flight per thread; the last
// block to finish reduces the per-block partials and writes the header (no
// second launch, no host round trip).  RANGE_THREADS threads per block.
__device__ void range_block(const float *__restrict__ x, unsigned long long n, int vec, RangePartial *partials,
                            unsigned int *counter, interp_header *hdr, Dims d, double eb, const interp_config &cfg,
                            double alpha, float *out_range, int b, int nb)
{
    float lo = INFINITY, hi = -INFINITY;
    unsigned long long bad = 0;
    const unsigned long long tid = (unsigned long long)b * RANGE_THREADS + threadIdx.x;
    const unsigned long long nthreads = (unsigned long long)nb * RANGE_THREADS;
    unsigned long long done = 0;
    if (vec) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const unsigned long long n4 = n / 4;
        unsigned long long i = tid;
        for (; i + 3 * nthreads < n4; i += 4 * nthreads) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = __ldcs(x4 + i + k * nthreads);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                range_acc(v[k].x, lo, hi, bad);
                range_acc(v[k].y, lo, hi, bad);
                range_acc(v[k].z, lo, hi, bad);
                range_acc(v[k].w, lo, hi, bad);
            }
        }
        for (; i < n4; i += nthreads) {
            const float4 v = __ldcs(x4 + i);
            range_acc(v.x, lo, hi, bad);
            range_acc(v.y, lo, hi, bad);
            range_acc(v.z, lo, hi, bad);
            range_acc(v.w, lo, hi, bad);
        }
        done = n4 * 4;
    }
    for (unsigned long long i = done + tid; i < n; i += nthreads) range_acc(__ldg(x + i), lo, hi, bad);

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
        bad += __shfl_xor_sync(0xffffffffu, bad, off);
    }
    __shared__ RangePartial warp_part[RANGE_THREADS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = RangePartial{lo, hi, bad};
    __syncthreads();
    if (threadIdx.x == 0) {
        RangePartial p = warp_part[0];
        for (int w = 1; w < RANGE_THREADS / 32; ++w) {
            p.lo = fminf(p.lo, warp_part[w].lo);
            p.hi = fmaxf(p.hi, warp_part[w].hi);
            p.nonfinite += warp_part[w].nonfinite;
        }
        partials[b] = p;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned int)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    lo = INFINITY;
    hi = -INFINITY;
    bad = 0;
    for (int k = threadIdx.x; k < nb; k += RANGE_THREADS) {
        const RangePartial p = partials[k];
        lo = fminf(lo, p.lo);
        hi = fmaxf(hi, p.hi);
        bad += p.nonfinite;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
        bad += __shfl_xor_sync(0xffffffffu, bad, off);
    }
    __syncthreads();
    if (lane == 0) warp_part[warp] = RangePartial{lo, hi, bad};
    __syncthreads();
    if (threadIdx.x == 0) {
        RangePartial p = warp_part[0];
        for (int w = 1; w < RANGE_THREADS / 32; ++w) {
            p.lo = fminf(p.lo, warp_part[w].lo);
            p.hi = fmaxf(p.hi, warp_part[w].hi);
            p.nonfinite += warp_part[w].nonfinite;
        }
        if (p.lo > p.hi) {  // no finite value at all
            p.lo = 0.0f;
            p.hi = 0.0f;
        }
        if (hdr) {
            write_bounds(hdr, d, eb, cfg, alpha, p.lo, p.hi, p.nonfinite);
        } else {
            out_range[0] = p.lo;
            out_range[1] = p.hi;
        }
        *counter = 0u;  // ready for the next call on this workspace
    }
}

__global__ void __launch_bounds__(RANGE_THREADS) k_range(const float *__restrict__ x, unsigned long long n, int vec,
                                                        RangePartial *partials, unsigned int *counter,
                                                        interp_header *hdr, Dims d, double eb, interp_config cfg,
                                                        double alpha, float *out_range)
{
    range_block(x, n, vec, partials, counter, hdr, d, eb, cfg, alpha, out_range, blockIdx.x, gridDim.x);
}

// ----------------------------------------------------- sampling profile
// Sample coordinate j (0..3) along an axis of length n: a uniform 4-point
// grid kept 12 points (or half the axis) away from both ends.
__device__ __forceinline__ int sample_coord(int n, int j)
{
    const int lo = min(12, (n - 1) / 2);
    return lo + j * (n - 1 - 2 * lo) / 3;
}

constexpr int PROFILE_SAMPLES = 64;

// Per sample and axis, with ORIGINAL neighbours at stride 1 and 2:
//   |x - NAK cubic|, |x - natural cubic|, |x - linear|,
//   2 |x - linear (stride 2)|, |x - quad-left (stride 2)| + |x - quad-right (stride 2)|.
// Sums per (axis, term) in sample order (z, y, x ascending), in double.
// The first 3 * PROFILE_SAMPLES threads of the block compute; every thread of
// the block takes part in its barriers.
__device__ void profile_block(const float *__restrict__ x, Dims d, interp_header *hdr, int apply, int first_axis)
{
    __shared__ double terms[3][5][PROFILE_SAMPLES];
    __shared__ double prof[18];
    const int t = threadIdx.x;
    const bool worker = t < 3 * PROFILE_SAMPLES;
    const int axis = worker ? t / PROFILE_SAMPLES : 0, smp = t % PROFILE_SAMPLES;
    const int n3[3] = {d.nz, d.ny, d.nx};
    const long long st[3] = {(long long)d.ny * d.nx, (long long)d.nx, 1};
    const int c[3] = {sample_coord(d.nz, smp / 16), sample_coord(d.ny, (smp / 4) % 4), sample_coord(d.nx, smp % 4)};
    const long long i = ((long long)c[0] * d.ny + c[1]) * d.nx + c[2];
    const int n = c[axis], nd = n3[axis];
    const long long sd = st[axis];
    const double xv = (double)x[i];
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0;
    const bool chunked = worker && axis >= first_axis;  // the leading axes of 1-D / 2-D data are not profiled
    if (chunked && n - 3 >= 0 && n + 3 <= nd - 1) {
        const float m3 = x[i - 3 * sd], m1 = x[i - sd], p1 = x[i + sd], p3 = x[i + 3 * sd];
        t0 = fabs(xv - (double)sp_cubic(cubic_coeffs(0), m3, m1, p1, p3));
        t1 = fabs(xv - (double)sp_cubic(cubic_coeffs(1), m3, m1, p1, p3));
    }
    if (chunked && n - 1 >= 0 && n + 1 <= nd - 1) t2 = fabs(xv - (double)sp_linear(x[i - sd], x[i + sd]));
    if (chunked && n - 6 >= 0 && n + 6 <= nd - 1) {
        const float m3 = x[i - 6 * sd], m1 = x[i - 2 * sd], p1 = x[i + 2 * sd], p3 = x[i + 6 * sd];
        t3 = 2.0 * fabs(xv - (double)sp_linear(m1, p1));
        t4 = fabs(xv - (double)sp_quad_left(m3, m1, p1)) + fabs(xv - (double)sp_quad_right(m1, p1, p3));
    }
    if (worker) {
        terms[axis][0][smp] = t0;
        terms[axis][1][smp] = t1;
        terms[axis][2][smp] = t2;
        terms[axis][3][smp] = t3;
        terms[axis][4][smp] = t4;
    }
    __syncthreads();
    if (t < 15) {
        const int a = t % 3, term = t / 3;
        double s = 0.0;
        for (int k = 0; k < PROFILE_SAMPLES; ++k) s += terms[a][term][k];
        // slots: 3a+0 NAK, 3a+1 natural, 9+a linear, 12+a linear s2, 15+a quadratic s2
        const int slot = term < 2 ? 3 * a + term : 9 + 3 * (term - 2) + a;
        prof[slot] = s;
    } else if (t < 18) {
        prof[3 * (t - 15) + 2] = 0.0;
    }
    __syncthreads();
    if (t != 0) return;
    for (int k = 0; k < 18; ++k) hdr->profile[k] = prof[k];
    if (!apply) return;
    // Decision (Sec. IV-B.2): cubic with the lower error per axis (not-a-knot on
    // ties); axes by descending error of their cubic, ties to the lower axis id;
    // per level, linear only if strictly better than the splines.
    double err[3];
    int ck[3];
    for (int a = 0; a < 3; ++a) {
        ck[a] = prof[3 * a + 1] < prof[3 * a + 0] ? 1 : 0;
        err[a] = prof[3 * a + ck[a]];
    }
    // repeatedly take the first remaining axis of maximal error
    int ord[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a) {
        int best = a;
        for (int b = a + 1; b < 3; ++b)
            if (err[ord[b]] > err[ord[best]]) best = b;
        const int pick = ord[best];
        for (int b = best; b > a; --b) ord[b] = ord[b - 1];
        ord[a] = pick;
    }
    for (int a = 0; a < 3; ++a) {
        hdr->cfg.dim_order[a] = ord[a];
        hdr->cfg.cubic_kind[a] = ck[a];
    }
    const double spline1 = err[0] + err[1] + err[2];
    const double lin1 = prof[9] + prof[10] + prof[11];
    const double lin2 = prof[12] + prof[13] + prof[14];
    const double quad2 = prof[15] + prof[16] + prof[17];
    hdr->cfg.level_kind[0] = lin1 < spline1 ? 0 : 1;
    hdr->cfg.level_kind[1] = lin2 < quad2 ? 0 : 1;
    hdr->cfg.level_kind[2] = 1;
}

__global__ void __launch_bounds__(3 * PROFILE_SAMPLES) k_profile(const float *__restrict__ x, Dims d,
                                                                interp_header *hdr, int apply, int first_axis)
{
    profile_block(x, d, hdr, apply, first_axis);
}

// The set-up of compression for every field of a call in one launch: per field,
// a block for the sampling profile and decision (when autotuning), then the
// blocks of its value range and bounds (relative mode) or one block writing the
// bounds (absolute mode).  The profile writes only the header's profile and
// decided configuration, the bounds only the other fields, so they may run
// concurrently.
struct PrologueField {
    const float *x;
    unsigned long long n;
    int vec;
    RangePartial *partials;
    unsigned int *counter;
    interp_header *hdr;
    Dims d;
    double eb;
    interp_config cfg;
    double alpha;
    int first_axis;
    int b0;        // first block of the field
    int nprof;     // 1 when autotuning, else 0
    int nrange;    // range blocks (relative mode), or 1 (absolute mode)
};

struct PrologueBatch {
    PrologueField f[kMaxBatch];
    int n;
};

__global__ void __launch_bounds__(RANGE_THREADS) k_prologue(const __grid_constant__ PrologueBatch B)
{
    const int b = blockIdx.x;
    int fi = 0;
    while (fi + 1 < B.n && B.f[fi + 1].b0 <= b) ++fi;
    const PrologueField &F = B.f[fi];
    const int lb = b - F.b0;
    if (lb < F.nprof) {
        profile_block(F.x, F.d, F.hdr, 1, F.first_axis);
        return;
    }
    if (F.cfg.eb_mode)
        range_block(F.x, F.n, F.vec, F.partials, F.counter, F.hdr, F.d, F.eb, F.cfg, F.alpha, nullptr,
                    lb - F.nprof, F.nrange);
    else if (threadIdx.x == 0)
        write_bounds(F.hdr, F.d, F.eb, F.cfg, F.alpha, 0.0f, 0.0f, 0ull);
}

// Zero the parts of every field's workspace that must start at zero (control
// words, outlier block counters) and its histogram, one block per field.
struct ZeroField {
    uint32_t *ctrl;
    int ctrl_words;
    uint32_t *blockcnt;
    int nblk;
    uint32_t *hist;
    int bins;
};

struct ZeroBatch {
    ZeroField f[kMaxBatch];
    int n;
};

__global__ void __launch_bounds__(512) k_zero(const __grid_constant__ ZeroBatch B)
{
    const ZeroField &F = B.f[blockIdx.x];
    for (int i = threadIdx.x; i < F.ctrl_words; i += 512) F.ctrl[i] = 0u;
    for (int i = threadIdx.x; i < F.nblk; i += 512) F.blockcnt[i] = 0u;
    if (F.hist)
        for (int i = threadIdx.x; i < F.bins; i += 512) F.hist[i] = 0u;
}

}  // namespace

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
    return sms;
}

namespace {

// Blocks of a grid-stride range kernel that are resident at once on this
// device (one wave): a block that had to wait for a free slot would finish its
// whole share late.  Cached per device and kernel.
constexpr int kMaxRangeDevices = 64;
template <typename K>
int one_wave(K kernel, int *cache)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    if (dev >= 0 && dev < kMaxRangeDevices && cache[dev] > 0) return cache[dev];
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, RANGE_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int b = std::min(per_sm * sm_count(), RANGE_MAX_BLOCKS);
    if (dev >= 0 && dev < kMaxRangeDevices) cache[dev] = b;
    return b;
}
int range_wave[kMaxRangeDevices], prologue_wave[kMaxRangeDevices];

}  // namespace

int range_blocks() { return one_wave(k_range, range_wave); }

size_t range_partials_bytes() { return sizeof(RangePartial) * RANGE_MAX_BLOCKS; }

cudaError_t launch_header_init(interp_header *hdr, Dims d, double eb, interp_config cfg, double alpha,
                               cudaStream_t s)
{
    k_header_init<<<1, 32, 0, s>>>(hdr, d, eb, cfg, alpha);
    return cudaGetLastError();
}

cudaError_t launch_range(const float *x, Dims d, double eb, interp_config cfg, double alpha, interp_header *hdr,
                         void *partials, unsigned int *counter, int nblocks, cudaStream_t s, float *out_range)
{
    const unsigned long long n = (unsigned long long)d.nz * d.ny * d.nx;
    const int vec = (reinterpret_cast<uintptr_t>(x) % 16) == 0;
    if (nblocks > RANGE_MAX_BLOCKS) nblocks = RANGE_MAX_BLOCKS;
    k_range<<<nblocks, RANGE_THREADS, 0, s>>>(x, n, vec, reinterpret_cast<RangePartial *>(partials), counter, hdr, d,
                                             eb, cfg, alpha, out_range);
    return cudaGetLastError();
}

cudaError_t launch_prologue(const PrologueItem *items, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    PrologueBatch B;
    std::memset(&B, 0, sizeof(B));
    ZeroBatch Z;
    std::memset(&Z, 0, sizeof(Z));
    int blocks = 0;
    for (int i = 0; i < n; ++i) {
        const PrologueItem &it = items[i];
        PrologueField &F = B.f[i];
        F.x = it.x;
        F.d = it.d;
        F.n = (unsigned long long)it.d.nz * it.d.ny * it.d.nx;
        F.vec = (reinterpret_cast<uintptr_t>(it.x) % 16) == 0;
        F.partials = reinterpret_cast<RangePartial *>(it.partials);
        F.counter = it.counter;
        F.hdr = it.hdr;
        F.eb = it.eb;
        F.cfg = it.cfg;
        F.alpha = it.alpha;
        F.first_axis = (it.cfg.ndim == 1 || it.cfg.ndim == 2) ? 3 - it.cfg.ndim : 0;
        F.b0 = blocks;
        F.nprof = it.cfg.autotune ? 1 : 0;
        // range blocks: about 32 K values each, at most one wave beside the profile block
        const unsigned long long want = (F.n + 32767) / 32768;
        const int wave = std::max(1, one_wave(k_prologue, prologue_wave) - F.nprof);
        F.nrange = it.cfg.eb_mode ? (int)std::max(1ull, std::min<unsigned long long>(want, wave)) : 1;
        blocks += F.nprof + F.nrange;
        ZeroField &zf = Z.f[i];
        zf.ctrl = it.counter;
        zf.ctrl_words = it.ctrl_words;
        zf.blockcnt = it.blockcnt;
        zf.nblk = it.nblk;
        zf.hist = it.hist;
        zf.bins = 2 * it.cfg.radius;
    }
    B.n = n;
    Z.n = n;
    k_zero<<<n, 512, 0, s>>>(Z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_prologue<<<blocks, RANGE_THREADS, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_profile(const float *x, Dims d, interp_header *hdr, int apply_decision, cudaStream_t s, int ndim)
{
    const int first_axis = (ndim == 1 || ndim == 2) ? 3 - ndim : 0;
    k_profile<<<1, 3 * PROFILE_SAMPLES, 0, s>>>(x, d, hdr, apply_decision, first_axis);
    return cudaGetLastError();
}

}  // namespace gi
