// Quality report of a compression (Sec. IV-D, Fig. 4 and the PSNR comparison
// that follows it): statistics of the quant-code histogram (Shannon entropy
// in bits per point, the rate an entropy coder approaches; the number of
// nonzero quant-codes, i.e. points whose prediction error exceeded the bound)
// and the reconstruction error (sum of squares, maximum, PSNR over the value
// range).  Not part of the compression path; used to report what the codes
// and reconstructions of a run look like.
#include <cfloat>

#include "common.cuh"

namespace gi {
namespace {

constexpr int HQ_THREADS = 1024;
constexpr int EQ_THREADS = 512;
constexpr int EQ_MAX_BLOCKS = 1024;

struct ErrPartial {
    double sse, maxerr;
    float lo, hi;
    unsigned long long finite;
};

// One CTA over the 2R bins: counts, entropy (double, bins in ascending order
// per thread, then a fixed tree), largest |q| among kept codes.
__global__ void __launch_bounds__(HQ_THREADS) k_hist_stats(const uint32_t *__restrict__ hist, int radius,
                                                           interp_quality *out, int has_err)
{
    __shared__ double s_plogp[HQ_THREADS / 32];
    __shared__ unsigned long long s_n[HQ_THREADS / 32], s_nz[HQ_THREADS / 32];
    __shared__ int s_maxq[HQ_THREADS / 32];
    __shared__ unsigned long long n_total;
    const int bins = 2 * radius;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pass 1: totals
    unsigned long long n = 0, nz = 0;
    int maxq = 0;
    for (int c = threadIdx.x; c < bins; c += HQ_THREADS) {
        const uint32_t h = hist[c];
        n += h;
        if (c != radius) nz += h;  // nonzero quant-codes, outliers included
        if (h && c != 0 && c != radius) maxq = max(maxq, abs(c - radius));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, off);
        nz += __shfl_xor_sync(0xffffffffu, nz, off);
        maxq = max(maxq, __shfl_xor_sync(0xffffffffu, maxq, off));
    }
    if (lane == 0) {
        s_n[warp] = n;
        s_nz[warp] = nz;
        s_maxq[warp] = maxq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tn = 0, tz = 0;
        int tq = 0;
        for (int w = 0; w < HQ_THREADS / 32; ++w) {
            tn += s_n[w];
            tz += s_nz[w];
            tq = max(tq, s_maxq[w]);
        }
        n_total = tn;
        out->n = tn;
        out->n_outliers = hist[0];
        out->n_nonzero = tz;
        out->max_abs_q = tq;
        out->reserved = 0;
        if (!has_err) {
            out->n_finite = 0;
            out->sse = out->max_abs_err = out->vmin = out->vmax = out->psnr_db = nan("");
        }
    }
    __syncthreads();
    // pass 2: entropy H = -sum p log2 p, p = h / n
    const double inv_n = n_total ? 1.0 / (double)n_total : 0.0;
    double acc = 0.0;
    for (int c = threadIdx.x; c < bins; c += HQ_THREADS) {
        const uint32_t h = hist[c];
        if (h) {
            const double p = (double)h * inv_n;
            acc -= p * log2(p);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) s_plogp[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < HQ_THREADS / 32; ++w) t += s_plogp[w];
        out->entropy_bits = t;
    }
}

// Reconstruction error over the finite points of x: grid-stride partials,
// the last CTA to finish folds them and writes the report.
__global__ void __launch_bounds__(EQ_THREADS) k_err_stats(const float *__restrict__ x, const float *__restrict__ xr,
                                                          unsigned long long n, ErrPartial *partials,
                                                          unsigned int *counter, interp_quality *out)
{
    double sse = 0.0, maxerr = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    unsigned long long fin = 0;
    const unsigned long long tid = (unsigned long long)blockIdx.x * EQ_THREADS + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * EQ_THREADS;
    for (unsigned long long i = tid; i < n; i += nth) {
        const float a = __ldg(x + i);
        if (!(fabsf(a) <= FLT_MAX)) continue;  // non-finite values are stored exactly
        const float b = __ldg(xr + i);
        const double d = (double)a - (double)b;
        sse += d * d;
        maxerr = fmax(maxerr, fabs(d));
        lo = fminf(lo, a);
        hi = fmaxf(hi, a);
        ++fin;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sse += __shfl_xor_sync(0xffffffffu, sse, off);
        maxerr = fmax(maxerr, __shfl_xor_sync(0xffffffffu, maxerr, off));
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
        fin += __shfl_xor_sync(0xffffffffu, fin, off);
    }
    __shared__ ErrPartial wp[EQ_THREADS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wp[warp] = ErrPartial{sse, maxerr, lo, hi, fin};
    __syncthreads();
    if (threadIdx.x == 0) {
        ErrPartial p = wp[0];
        for (int w = 1; w < EQ_THREADS / 32; ++w) {
            p.sse += wp[w].sse;
            p.maxerr = fmax(p.maxerr, wp[w].maxerr);
            p.lo = fminf(p.lo, wp[w].lo);
            p.hi = fmaxf(p.hi, wp[w].hi);
            p.finite += wp[w].finite;
        }
        partials[blockIdx.x] = p;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    ErrPartial t = partials[0];
    for (unsigned b = 1; b < gridDim.x; ++b) {  // fixed order: reproducible for a given grid
        const ErrPartial p = partials[b];
        t.sse += p.sse;
        t.maxerr = fmax(t.maxerr, p.maxerr);
        t.lo = fminf(t.lo, p.lo);
        t.hi = fmaxf(t.hi, p.hi);
        t.finite += p.finite;
    }
    out->n_finite = t.finite;
    out->sse = t.sse;
    out->max_abs_err = t.maxerr;
    out->vmin = t.finite ? t.lo : nan("");
    out->vmax = t.finite ? t.hi : nan("");
    const double range = (double)t.hi - (double)t.lo;
    out->psnr_db = (t.finite && t.sse > 0.0) ? 20.0 * log10(range) - 10.0 * log10(t.sse / (double)t.finite)
                                             : (t.finite ? INFINITY : nan(""));
    *counter = 0u;
}

}  // namespace

size_t quality_workspace_bytes() { return 256 + sizeof(ErrPartial) * EQ_MAX_BLOCKS; }

cudaError_t launch_quality(const uint32_t *hist, int radius, const float *x, const float *xr, uint64_t n,
                           interp_quality *out, void *ws, cudaStream_t s)
{
    const int has_err = x && xr && n > 0;
    k_hist_stats<<<1, HQ_THREADS, 0, s>>>(hist, radius, out, has_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !has_err) return e;
    unsigned char *w = static_cast<unsigned char *>(ws);
    unsigned int *counter = reinterpret_cast<unsigned int *>(w);
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    unsigned long long blocks = (n + EQ_THREADS * 16ull - 1) / (EQ_THREADS * 16ull);
    const unsigned long long cap = (unsigned long long)min(EQ_MAX_BLOCKS, 4 * sm_count());
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_err_stats<<<(unsigned)blocks, EQ_THREADS, 0, s>>>(x, xr, (unsigned long long)n,
                                                        reinterpret_cast<ErrPartial *>(w + 256), counter, out);
    return cudaGetLastError();
}

}  // namespace gi
