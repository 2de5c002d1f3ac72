// G-Interp tile kernels: fused predict-quantize (compression) and the
// reconstruction replay (decompression), Sec. IV-A/B/C of arXiv 2312.05492.
//
// One CTA owns a tile of TZ x TY x TX chunks of 8^3 points.  Because every
// interpolation stays inside the closed 8^3 chunk along its axis (anchors
// "bound" the interpolation, Sec. IV-A), a tile depends only on the original
// values of its box = owned points + the closing faces at the far end of
// each axis.  The CTA stages that box in shared memory, recomputes the
// far-face points (bit-identical to what the neighbouring tile computes for
// them), and runs the nine dependent passes (strides 4, 2, 1; three axes
// each, Sec. IV-A) with a barrier between passes.
//
// Work unit inside a pass: one chunk segment, i.e. the 9 points of one line
// along the pass axis inside one chunk.  Its known points (even multiples of
// s) give every prediction of the segment (1, 2 or 4 of them) from registers:
// the full-chunk stencils are fixed (Fig. 3); chunks truncated by the field's
// far edge take the neighbour-count rule point by point.
#include "common.cuh"

namespace gi {
namespace {

__host__ __device__ constexpr int box_ext(int a) { return a == 2 ? BX : (a == 1 ? BY : BZ); }
__host__ __device__ constexpr int own_ext(int a) { return a == 2 ? OX : (a == 1 ? OY : OZ); }
__host__ __device__ constexpr int box_stride(int a) { return a == 2 ? 1 : (a == 1 ? BX : BX * BY); }
__host__ __device__ constexpr int own_stride(int a) { return a == 2 ? 1 : (a == 1 ? OX : OX * OY); }
__host__ __device__ constexpr int chunks_of(int a) { return a == 2 ? TX : (a == 1 ? TY : TZ); }
// the two axes other than d: U is the faster-varying one in memory
__host__ __device__ constexpr int axis_u(int d) { return d == 2 ? 1 : 2; }
__host__ __device__ constexpr int axis_v(int d) { return d == 0 ? 1 : 0; }
__host__ __device__ constexpr int rank_in(int a, int o0, int o1, int o2) { return a == o0 ? 0 : (a == o1 ? 1 : 2); }

// dynamic shared-memory layout; every sub-array starts on a 16-byte boundary
__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) / 16 * 16; }
constexpr size_t kCompressCodesOff = align16(sizeof(float) * BOX);
constexpr size_t kCompressHistOff = align16(kCompressCodesOff + sizeof(uint16_t) * OWN);
constexpr size_t kCompressSmem = kCompressHistOff + sizeof(uint32_t) * HIST_SMEM_BINS;
constexpr size_t kDecompressCodesOff = align16(sizeof(float) * BOX);
constexpr size_t kDecompressSmem = kDecompressCodesOff + sizeof(uint16_t) * BOX;
static_assert(kCompressCodesOff % 16 == 0 && (sizeof(uint16_t) * OX) % 16 == 0, "uint4 access to owned code rows");

struct TileCtx {
    int g0[3];  // global origin of the tile (z, y, x)
    int n[3];   // field dims
    LevelQ L[3];
    int R;
    float Rf;
    int spline[3];  // per level
    Cubic cub[3];   // per axis
};

struct CompressSink {
    uint16_t *own_codes;  // [OZ][OY][OX]
    uint32_t *hist_s;     // shared bins or null
    uint32_t *hist_g;     // global bins (used when hist_s is null); may be null
    uint32_t central;     // register count of code R
};

// One pass (level S, axis D).  U_EARLY / V_EARLY: whether the other axes come
// before D in the dim order (then they are on the s-grid, else on the 2s-grid).
template <bool COMPRESS, int S, int D, bool U_EARLY, bool V_EARLY>
__device__ __forceinline__ void run_pass(float *__restrict__ box, uint16_t *__restrict__ cbox, const TileCtx &c,
                                         CompressSink &sink)
{
    constexpr int U = axis_u(D), V = axis_v(D);
    constexpr int stepU = U_EARLY ? S : 2 * S;
    constexpr int stepV = V_EARLY ? S : 2 * S;
    constexpr int nU = (box_ext(U) - 1) / stepU + 1;
    constexpr int nV = (box_ext(V) - 1) / stepV + 1;
    constexpr int nC = chunks_of(D);
    constexpr int NSEG = nU * nV * nC;
    constexpr int SD = box_stride(D), SU = box_stride(U), SV = box_stride(V);
    constexpr int OD = own_stride(D), OU = own_stride(U), OV = own_stride(V);
    constexpr int l = S == 1 ? 0 : (S == 2 ? 1 : 2);

    const LevelQ Lq = c.L[l];
    const bool spline = c.spline[l] != 0;
    const Cubic cub = c.cub[D];
    const int R = c.R;
    const float Rf = c.Rf;

    for (int w = threadIdx.x; w < NSEG; w += TILE_THREADS) {
        int iu, iv, cd;
        if (D == 2) {
            cd = w % nC;
            const int r = w / nC;
            iu = r % nU;
            iv = r / nU;
        } else {
            iu = w % nU;
            const int r = w / nU;
            cd = r % nC;
            iv = r / nC;
        }
        const int u = iu * stepU, v = iv * stepV, dlo = 8 * cd;
        const int gd = c.g0[D] + dlo;
        if (c.g0[U] + u >= c.n[U] || c.g0[V] + v >= c.n[V] || gd + S > c.n[D] - 1) continue;
        const bool owned = (u < own_ext(U)) && (v < own_ext(V));
        float *line = box + v * SV + u * SU + dlo * SD;
        const int lbox = v * SV + u * SU + dlo * SD;
        const int lown = v * OV + u * OU + dlo * OD;

        auto emit = [&](int o, float p) {
            if (COMPRESS) {
                const float x = line[o * SD];
                float xr;
                const uint32_t code = quantize(x, p, Lq, R, Rf, xr);
                line[o * SD] = xr;
                if (owned) {
                    sink.own_codes[lown + o * OD] = (uint16_t)code;
                    if (code == (uint32_t)R) {
                        sink.central++;
                    } else if (sink.hist_s) {
                        atomicAdd(&sink.hist_s[code], 1u);
                    } else if (sink.hist_g) {
                        atomicAdd(&sink.hist_g[code], 1u);
                    }
                }
            } else {
                const uint32_t code = cbox[lbox + o * SD];
                line[o * SD] = dequantize(code, p, Lq, R, line[o * SD]);
            }
        };

        const int hi = min(8, c.n[D] - 1 - gd);  // last offset of the (possibly truncated) chunk
        if (hi == 8) {
            if (S == 4) {
                emit(4, sp_linear(line[0], line[8 * SD]));
            } else if (S == 2) {
                const float k0 = line[0], k4 = line[4 * SD], k8 = line[8 * SD];
                if (spline) {
                    emit(2, sp_quad_right(k0, k4, k8));
                    emit(6, sp_quad_left(k0, k4, k8));
                } else {
                    emit(2, sp_linear(k0, k4));
                    emit(6, sp_linear(k4, k8));
                }
            } else {
                const float k0 = line[0], k2 = line[2 * SD], k4 = line[4 * SD], k6 = line[6 * SD],
                            k8 = line[8 * SD];
                if (spline) {
                    emit(1, sp_quad_right(k0, k2, k4));
                    emit(3, sp_cubic(cub, k0, k2, k4, k6));
                    emit(5, sp_cubic(cub, k2, k4, k6, k8));
                    emit(7, sp_quad_left(k4, k6, k8));
                } else {
                    emit(1, sp_linear(k0, k2));
                    emit(3, sp_linear(k2, k4));
                    emit(5, sp_linear(k4, k6));
                    emit(7, sp_linear(k6, k8));
                }
            }
        } else {
            // chunk truncated by the far edge of the field: neighbour-count rule
#pragma unroll
            for (int o = S; o < 8; o += 2 * S) {
                if (o > hi) break;
                const bool has_m3 = o - 3 * S >= 0;
                const bool has_p1 = o + S <= hi;
                const bool has_p3 = o + 3 * S <= hi;
                const float m1 = line[(o - S) * SD];
                float p;
                if (!has_p1) {
                    p = m1;
                } else {
                    const float p1 = line[(o + S) * SD];
                    if (!spline) {
                        p = sp_linear(m1, p1);
                    } else if (has_m3 && has_p3) {
                        p = sp_cubic(cub, line[(o - 3 * S) * SD], m1, p1, line[(o + 3 * S) * SD]);
                    } else if (has_m3) {
                        p = sp_quad_left(line[(o - 3 * S) * SD], m1, p1);
                    } else if (has_p3) {
                        p = sp_quad_right(m1, p1, line[(o + 3 * S) * SD]);
                    } else {
                        p = sp_linear(m1, p1);
                    }
                }
                emit(o, p);
            }
        }
    }
}

template <bool COMPRESS, int O0, int O1, int O2, int S>
__device__ __forceinline__ void run_level(float *box, uint16_t *cbox, const TileCtx &c, CompressSink &sink)
{
    // pass k = 0: both other axes come later; k = 2: both earlier; k = 1: one each
    run_pass<COMPRESS, S, O0, false, false>(box, cbox, c, sink);
    __syncthreads();
    run_pass<COMPRESS, S, O1, rank_in(axis_u(O1), O0, O1, O2) < 1, rank_in(axis_v(O1), O0, O1, O2) < 1>(box, cbox,
                                                                                                      c, sink);
    __syncthreads();
    run_pass<COMPRESS, S, O2, true, true>(box, cbox, c, sink);
    __syncthreads();
}

template <bool COMPRESS, int O0, int O1, int O2>
__device__ __forceinline__ void run_levels(float *box, uint16_t *cbox, const TileCtx &c, CompressSink &sink)
{
    run_level<COMPRESS, O0, O1, O2, 4>(box, cbox, c, sink);
    run_level<COMPRESS, O0, O1, O2, 2>(box, cbox, c, sink);
    run_level<COMPRESS, O0, O1, O2, 1>(box, cbox, c, sink);
}

template <bool COMPRESS>
__device__ void dispatch_order(int oid, float *box, uint16_t *cbox, const TileCtx &c, CompressSink &sink)
{
    switch (oid) {
    case 0: run_levels<COMPRESS, 0, 1, 2>(box, cbox, c, sink); break;
    case 1: run_levels<COMPRESS, 0, 2, 1>(box, cbox, c, sink); break;
    case 2: run_levels<COMPRESS, 1, 0, 2>(box, cbox, c, sink); break;
    case 3: run_levels<COMPRESS, 1, 2, 0>(box, cbox, c, sink); break;
    case 4: run_levels<COMPRESS, 2, 0, 1>(box, cbox, c, sink); break;
    default: run_levels<COMPRESS, 2, 1, 0>(box, cbox, c, sink); break;
    }
}

__device__ __forceinline__ int order_id(const int32_t o[3])
{
    // lexicographic rank of the permutation
    if (o[0] == 0) return o[1] == 1 ? 0 : 1;
    if (o[0] == 1) return o[1] == 0 ? 2 : 3;
    return o[1] == 0 ? 4 : 5;
}

__device__ __forceinline__ void tile_setup(TileCtx &c, const interp_header *hdr, Dims d, int b, int tiles_y,
                                           int tiles_x)
{
    const int tx = b % tiles_x;
    const int ty = (b / tiles_x) % tiles_y;
    const int tz = b / (tiles_x * tiles_y);
    c.g0[0] = tz * OZ;
    c.g0[1] = ty * OY;
    c.g0[2] = tx * OX;
    c.n[0] = d.nz;
    c.n[1] = d.ny;
    c.n[2] = d.nx;
    for (int l = 0; l < 3; ++l) {
        c.L[l].e = hdr->e[l];
        c.L[l].twoe = hdr->twoe[l];
        c.L[l].inv2e = hdr->inv2e[l];
        c.spline[l] = hdr->cfg.level_kind[l];
        c.cub[l] = cubic_coeffs(hdr->cfg.cubic_kind[l]);
    }
    c.R = hdr->cfg.radius;
    c.Rf = (float)c.R;
}

// ------------------------------------------------------------ compression
__global__ void __launch_bounds__(TILE_THREADS) k_compress(CompressArgs a, TileGrid tg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *box = reinterpret_cast<float *>(smem);
    uint16_t *own_codes = reinterpret_cast<uint16_t *>(smem + kCompressCodesOff);  // 16-byte aligned rows
    uint32_t *hist_s = reinterpret_cast<uint32_t *>(smem + kCompressHistOff);

    TileCtx c;
    tile_setup(c, a.hdr, a.dims, blockIdx.x, tg.ty, tg.tx);
    const int nz = a.dims.nz, ny = a.dims.ny, nx = a.dims.nx;
    const int bins = 2 * c.R;
    const bool smem_hist = a.hist != nullptr && bins <= HIST_SMEM_BINS;
    if (smem_hist)
        for (int i = threadIdx.x; i < bins; i += TILE_THREADS) hist_s[i] = 0u;

    // ---- stage the box (owned points + far faces) of original values
    const bool vec = a.vec_x;
    for (int i = threadIdx.x; i < BZ * BY * (OX / 4); i += TILE_THREADS) {
        const int q = i % (OX / 4);
        const int row = i / (OX / 4);
        const int lz = row / BY, ly = row % BY;
        const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + 4 * q;
        if (gz >= nz || gy >= ny || gx >= nx) continue;
        const size_t gi = ((size_t)gz * ny + gy) * nx + gx;
        float *dst = box + (lz * BY + ly) * BX + 4 * q;
        if (vec) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(a.x + gi));
            dst[0] = v.x;
            dst[1] = v.y;
            dst[2] = v.z;
            dst[3] = v.w;
        } else {
            for (int j = 0; j < 4 && gx + j < nx; ++j) dst[j] = __ldg(a.x + gi + j);
        }
    }
    for (int row = threadIdx.x; row < BZ * BY; row += TILE_THREADS) {
        const int lz = row / BY, ly = row % BY;
        const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + OX;
        if (gz >= nz || gy >= ny || gx >= nx) continue;
        box[(lz * BY + ly) * BX + OX] = __ldg(a.x + ((size_t)gz * ny + gy) * nx + gx);
    }
    __syncthreads();

    CompressSink sink{own_codes, smem_hist ? hist_s : nullptr, a.hist, 0u};

    // ---- anchors owned by the tile: stored losslessly, code R (Sec. IV-A)
    {
        const int Ay = (ny - 1) / 8 + 1, Ax = (nx - 1) / 8 + 1;
        for (int i = threadIdx.x; i < TZ * TY * TX; i += TILE_THREADS) {
            const int ax = i % TX, ay = (i / TX) % TY, az = i / (TX * TY);
            const int lz = 8 * az, ly = 8 * ay, lx = 8 * ax;
            const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + lx;
            if (gz >= nz || gy >= ny || gx >= nx) continue;
            a.anchors[((size_t)(gz / 8) * Ay + gy / 8) * Ax + gx / 8] = box[(lz * BY + ly) * BX + lx];
            own_codes[(lz * OY + ly) * OX + lx] = (uint16_t)c.R;
            sink.central++;
        }
    }

    // ---- the nine passes
    dispatch_order<true>(order_id(a.hdr->cfg.dim_order), box, nullptr, c, sink);

    // ---- codes, outlier bitmap words and histogram
    const int words_per_row = (nx + 31) / 32;
    if (a.vec_codes) {
        // 4 lanes per owned row, 8 codes (16 bytes) per lane
        for (int i = threadIdx.x; i < OZ * OY * (OX / 8); i += TILE_THREADS) {
            const int sub = i % (OX / 8);
            const int row = i / (OX / 8);
            const int lz = row / OY, ly = row % OY;
            const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + 8 * sub;
            const bool in = gz < nz && gy < ny && gx < nx;
            uint32_t m = 0;
            if (in) {
                const uint4 v = *reinterpret_cast<const uint4 *>(own_codes + row * OX + 8 * sub);
                *reinterpret_cast<uint4 *>(a.codes + ((size_t)gz * ny + gy) * nx + gx) = v;
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    m |= (uint32_t)((w4[j] & 0xffffu) == 0u) << (2 * j);
                    m |= (uint32_t)((w4[j] >> 16) == 0u) << (2 * j + 1);
                }
            }
            // OX / 8 = 4 consecutive lanes form one 32-bit word
            uint32_t word = m << (8 * sub);
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            if (sub == 0 && gz < nz && gy < ny) {
                const int64_t wi = ((int64_t)gz * ny + gy) * words_per_row + c.g0[2] / 32;
                a.bitmap[wi] = word;
                if (word) atomicAdd(&a.blockcnt[wi / BITMAP_BLOCK_WORDS], (uint32_t)__popc(word));
            }
        }
    } else {
        // one warp per owned row of 32 x-positions
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int row = warp; row < OZ * OY * (OX / 32); row += TILE_THREADS / 32) {
            const int seg = row % (OX / 32);
            const int r = row / (OX / 32);
            const int lz = r / OY, ly = r % OY;
            const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + 32 * seg + lane;
            if (gz >= nz || gy >= ny) continue;  // warp-uniform
            const bool in = gx < nx;
            uint32_t code = 1;
            if (in) {
                code = own_codes[r * OX + 32 * seg + lane];
                a.codes[((size_t)gz * ny + gy) * nx + gx] = (uint16_t)code;
            }
            const uint32_t word = __ballot_sync(0xffffffffu, in && code == 0u);
            if (lane == 0 && c.g0[2] + 32 * seg < nx) {
                const int64_t wi = ((int64_t)gz * ny + gy) * words_per_row + (c.g0[2] + 32 * seg) / 32;
                a.bitmap[wi] = word;
                if (word) atomicAdd(&a.blockcnt[wi / BITMAP_BLOCK_WORDS], (uint32_t)__popc(word));
            }
        }
    }

    if (a.hist) {
        uint32_t cnt = sink.central;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if ((threadIdx.x & 31) == 0 && cnt) {
            if (smem_hist) atomicAdd(&hist_s[c.R], cnt);
            else atomicAdd(&a.hist[c.R], cnt);
        }
        if (smem_hist) {
            __syncthreads();
            for (int i = threadIdx.x; i < bins; i += TILE_THREADS) {
                const uint32_t h = hist_s[i];
                if (h) atomicAdd(&a.hist[i], h);
            }
        }
    }
}

// ---------------------------------------------------------- decompression
__global__ void __launch_bounds__(TILE_THREADS) k_decompress(DecompressArgs a, TileGrid tg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *box = reinterpret_cast<float *>(smem);
    uint16_t *cbox = reinterpret_cast<uint16_t *>(smem + kDecompressCodesOff);

    TileCtx c;
    tile_setup(c, a.hdr, a.dims, blockIdx.x, tg.ty, tg.tx);
    const int nz = a.dims.nz, ny = a.dims.ny, nx = a.dims.nx;

    // ---- stage quant-codes of the whole box; outlier values for code 0
    const bool vec = a.vec_codes;
    for (int i = threadIdx.x; i < BZ * BY * (OX / 8); i += TILE_THREADS) {
        const int q = i % (OX / 8);
        const int row = i / (OX / 8);
        const int lz = row / BY, ly = row % BY;
        const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + 8 * q;
        if (gz >= nz || gy >= ny || gx >= nx) continue;
        const size_t gi = ((size_t)gz * ny + gy) * nx + gx;
        const int li = (lz * BY + ly) * BX + 8 * q;
        if (vec) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.codes + gi));
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t c0 = w4[j] & 0xffffu, c1 = w4[j] >> 16;
                cbox[li + 2 * j] = (uint16_t)c0;
                cbox[li + 2 * j + 1] = (uint16_t)c1;
                if (c0 == 0u) box[li + 2 * j] = a.xrec[gi + 2 * j];
                if (c1 == 0u) box[li + 2 * j + 1] = a.xrec[gi + 2 * j + 1];
            }
        } else {
            for (int j = 0; j < 8 && gx + j < nx; ++j) {
                const uint16_t cj = __ldg(a.codes + gi + j);
                cbox[li + j] = cj;
                if (cj == 0) box[li + j] = a.xrec[gi + j];
            }
        }
    }
    for (int row = threadIdx.x; row < BZ * BY; row += TILE_THREADS) {
        const int lz = row / BY, ly = row % BY;
        const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + OX;
        if (gz >= nz || gy >= ny || gx >= nx) continue;
        const size_t gi = ((size_t)gz * ny + gy) * nx + gx;
        const uint16_t cj = __ldg(a.codes + gi);
        cbox[(lz * BY + ly) * BX + OX] = cj;
        if (cj == 0) box[(lz * BY + ly) * BX + OX] = a.xrec[gi];
    }
    // anchors of the box, including the borrowed ones on the far faces
    {
        const int Ay = (ny - 1) / 8 + 1, Ax = (nx - 1) / 8 + 1;
        for (int i = threadIdx.x; i < (TZ + 1) * (TY + 1) * (TX + 1); i += TILE_THREADS) {
            const int ax = i % (TX + 1), ay = (i / (TX + 1)) % (TY + 1), az = i / ((TX + 1) * (TY + 1));
            const int lz = 8 * az, ly = 8 * ay, lx = 8 * ax;
            const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + lx;
            if (gz >= nz || gy >= ny || gx >= nx) continue;
            box[(lz * BY + ly) * BX + lx] = __ldg(a.anchors + ((size_t)(gz / 8) * Ay + gy / 8) * Ax + gx / 8);
        }
    }
    __syncthreads();

    CompressSink sink{nullptr, nullptr, nullptr, 0u};
    dispatch_order<false>(order_id(a.hdr->cfg.dim_order), box, cbox, c, sink);

    // ---- write the owned reconstruction
    const bool vec4 = a.vec_xrec;
    for (int i = threadIdx.x; i < OZ * OY * (OX / 4); i += TILE_THREADS) {
        const int q = i % (OX / 4);
        const int row = i / (OX / 4);
        const int lz = row / OY, ly = row % OY;
        const int gz = c.g0[0] + lz, gy = c.g0[1] + ly, gx = c.g0[2] + 4 * q;
        if (gz >= nz || gy >= ny || gx >= nx) continue;
        const size_t gi = ((size_t)gz * ny + gy) * nx + gx;
        const float *src = box + (lz * BY + ly) * BX + 4 * q;
        if (vec4) {
            *reinterpret_cast<float4 *>(a.xrec + gi) = make_float4(src[0], src[1], src[2], src[3]);
        } else {
            for (int j = 0; j < 4 && gx + j < nx; ++j) a.xrec[gi + j] = src[j];
        }
    }
}


// The dynamic shared-memory opt-in is a per-device function attribute: set it
// once for every device the library is used on.
constexpr int kMaxDevices = 64;
volatile int compress_attr_done[kMaxDevices];
volatile int decompress_attr_done[kMaxDevices];

template <typename K>
cudaError_t ensure_smem_attr(K kernel, size_t bytes, volatile int *done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) done[dev] = 1;
    return e;
}

TileGrid tile_grid(Dims d)
{
    return TileGrid{(d.nz + OZ - 1) / OZ, (d.ny + OY - 1) / OY, (d.nx + OX - 1) / OX};
}

}  // namespace

cudaError_t launch_compress_tiles(const CompressArgs &a, cudaStream_t s)
{
    cudaError_t e = ensure_smem_attr(k_compress, kCompressSmem, compress_attr_done);
    if (e != cudaSuccess) return e;
    const TileGrid tg = tile_grid(a.dims);
    const long long n = (long long)tg.tz * tg.ty * tg.tx;
    if (n <= 0) return cudaSuccess;
    k_compress<<<(unsigned)n, TILE_THREADS, kCompressSmem, s>>>(a, tg);
    return cudaGetLastError();
}

cudaError_t launch_decompress_tiles(const DecompressArgs &a, cudaStream_t s)
{
    cudaError_t e = ensure_smem_attr(k_decompress, kDecompressSmem, decompress_attr_done);
    if (e != cudaSuccess) return e;
    const TileGrid tg = tile_grid(a.dims);
    const long long n = (long long)tg.tz * tg.ty * tg.tx;
    if (n <= 0) return cudaSuccess;
    k_decompress<<<(unsigned)n, TILE_THREADS, kDecompressSmem, s>>>(a, tg);
    return cudaGetLastError();
}

}  // namespace gi
