// G-Interp tile kernels: fused predict-quantize (compression) and the
// reconstruction replay (decompression), Sec. IV-A/B/C of arXiv 2312.05492.
//
// Decomposition.  Every interpolation stays inside the closed 8^3 chunk along
// its axis (anchors bound it, Sec. IV-A), so a column of 2 x 4 chunks
// (16 y x 32 x owned points) can be processed one 8-plane slab at a time: the
// slab's box is 9 planes x 17 rows x 33 columns (owned points plus the
// closing faces at the far end of each axis).  The face plane shared by two
// consecutive slabs depends only on values inside that plane, so it is
// computed once and carried to the next slab; the far row (y) and column (x)
// faces are recomputed by the neighbouring column (bit-identical values).
//
// Persistent CTAs take work items = (column, run of slabs) round-robin and
// march along z.  One thread issues a TMA box load of the next slab into a
// dense staging buffer while the CTA runs the nine dependent passes (strides
// 4, 2, 1; three axes each, a barrier between passes) on the current slab;
// the staging buffer is then repacked into the compute box, whose odd row
// pitch (33 floats) and plane pitch (561) make row-per-thread and
// column-per-thread walks free of shared-memory bank conflicts.
//
// Work unit inside a pass: one chunk segment, i.e. the 9 points of a line
// along the pass axis inside one chunk; its known points (even multiples of
// s) give all 1, 2 or 4 predictions of the segment from registers.
// Full-chunk stencils are fixed (Fig. 3); chunks truncated by the field's far
// edge take the neighbour-count rule point by point.
#include <algorithm>
#include <cstring>

#include "tma.cuh"

namespace gi {
namespace {

// ------------------------------------------------------------ geometry
constexpr int NT = TILE_THREADS;
constexpr int NWARP = NT / 32;
constexpr int EZ = 9, EY = OY + 1, EX = OX + 1;  // slab box extents (z, y, x)
constexpr int PLANE = EY * EX;                   // 561 floats, odd: conflict-free row walks
constexpr int BOXF = EZ * PLANE;                 // floats per slab box
constexpr int CP = OX + 2;                       // u16 pitch of code rows (17 words, odd)
constexpr int CBOX_PLANE = EY * CP;              // code box (compression staging, decompression input):
constexpr int CBOX = EZ * CBOX_PLANE;            // every row and column of the slab box
constexpr int STAGE_PLANE = CBOX_PLANE;
constexpr int STAGE = CBOX;
// TMA landing buffers: dense boxes whose rows are a multiple of 16 bytes
constexpr int XP = 36;                           // floats per landed row (x 0..35)
constexpr int XPL = 8;                           // landed input planes: 1..8 of a slab (plane 0 is
                                                 // carried, or loaded directly at a run's start)
constexpr int XLAND = XPL * EY * XP;
constexpr int KP = 40;                           // codes per landed row (x 0..39)
constexpr int KLAND = EZ * EY * KP;
constexpr uint32_t kTmaPolls = 1u << 22;         // bounded wait for one TMA box

__host__ __device__ constexpr int ext_of(int a) { return a == 2 ? EX : (a == 1 ? EY : EZ); }
__host__ __device__ constexpr int own_of(int a) { return a == 2 ? OX : (a == 1 ? OY : EZ); }
__host__ __device__ constexpr int bstride(int a) { return a == 2 ? 1 : (a == 1 ? EX : PLANE); }
__host__ __device__ constexpr int sstride(int a) { return a == 2 ? 1 : (a == 1 ? CP : STAGE_PLANE); }
__host__ __device__ constexpr int cstride(int a) { return a == 2 ? 1 : (a == 1 ? CP : CBOX_PLANE); }
// decompression reads the codes where the TMA landed them: rows of KP codes, planes of EY rows
__host__ __device__ constexpr int lstride(int a) { return a == 2 ? 1 : (a == 1 ? KP : EY * KP); }
static_assert((KP * 2) % 16 == 0, "landed code rows stay 16-byte aligned");
static_assert(KP == 5 * 8, "a landed code row is 5 groups of 8 codes");
__host__ __device__ constexpr int chunks_of(int a) { return a == 2 ? OX / 8 : (a == 1 ? OY / 8 : 1); }
__host__ __device__ constexpr int axis_u(int d) { return d == 2 ? 1 : 2; }  // faster other axis
__host__ __device__ constexpr int axis_v(int d) { return d == 0 ? 1 : 0; }
__host__ __device__ constexpr int count_on(int e, int step) { return (e - 1) / step + 1; }
__host__ __device__ constexpr uint32_t magic_of(int n)
{
    return n <= 1 ? 0u : (uint32_t)((0x100000000ull + (unsigned long long)n - 1) / (unsigned long long)n);
}

// floor(w / n) for 0 <= w < 2^16 and 1 <= n <= 64, given magic_of(n) (0 for n = 1)
__device__ __forceinline__ int fdiv(int w, uint32_t m) { return m ? (int)__umulhi((uint32_t)w, m) : w; }

// dynamic shared-memory layouts: the TMA landing buffer first (the dynamic
// shared-memory base is 128-byte aligned), then 16-byte aligned sub-arrays
__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) / 16 * 16; }
// compression: the staged codes reuse the landing buffer (the next slab's load is
// issued once they are written out)
constexpr size_t C_LAND = 0;
constexpr size_t C_STAGE = C_LAND;
constexpr size_t C_BOX = al16(C_LAND + sizeof(float) * XLAND);
constexpr size_t C_HIST = al16(C_BOX + sizeof(float) * BOXF);
// histogram bins, then one spare word per lane that takes the updates a point
// does not count (a predicated update would become a branch per point)
constexpr int HIST_WORDS = HIST_SMEM_BINS + 32;
constexpr size_t C_BAR = al16(C_HIST + sizeof(uint32_t) * HIST_WORDS);
constexpr size_t kCompressSmem = C_BAR + 16;
static_assert(sizeof(uint16_t) * STAGE <= sizeof(float) * XLAND, "staged codes fit the landing buffer");
// decompression: one code landing buffer (the next slab's codes land once the
// current slab's passes are done with theirs), then the value box and its barrier
__host__ __device__ constexpr size_t al128(size_t v) { return (v + 127) / 128 * 128; }
constexpr size_t D_LAND = 0;
constexpr size_t D_BOX = al128(sizeof(uint16_t) * KLAND);
constexpr size_t D_BAR = al16(D_BOX + sizeof(float) * BOXF);
constexpr size_t kDecompressSmem = D_BAR + 16;
// with 16-row columns, 5 compression CTAs fit an SM: dynamic + static (< 512 B) + 1 KB reserved each
constexpr int kCompressCtas = 5;
static_assert(OY != 16 || kCompressCtas * (kCompressSmem + 512 + 1024) <= 228 * 1024, "compression CTAs per SM");
// the smaller decompression CTA leaves room for six (at 56 registers a thread)
constexpr int kDecompressCtas = 6;
static_assert(OY != 16 || kDecompressCtas * (kDecompressSmem + 512 + 1024) <= 228 * 1024,
              "decompression CTAs per SM");

// Nonzero iff one of the two 16-bit halves of w is zero (a borrow can only set
// bits above a zero half, never create one).
__device__ __forceinline__ uint32_t has_zero_half(uint32_t w) { return (w - 0x00010001u) & ~w & 0x80008000u; }


// ------------------------------------------------------------ context
struct Field {
    int n[3];    // nz, ny, nx
    int cols_x;  // columns along x
    int cols;    // columns in total
    int slabs;   // slabs along z
    int run;     // slabs per work item
    int items;   // work items
};

struct Slab {
    int g0[3];           // global origin of the slab box (z, y, x)
    int col;             // column index (cy * cols_x + cx)
    bool carried;        // plane 0 carried from the previous slab (not recomputed)
    int own_lo, own_hi;  // local planes whose outputs this slab writes
    int lim[3];          // per axis: box positions below lim are owned and inside the field
                         // (z: planes up to own_hi; y, x: owned rows / columns)
};

// Per-call constants, one copy in shared memory.
struct Levels {
    LevelQ L[3];
    int spline[3];
    Cubic cub[3];
    int order[3];
    int rank[3];  // position of each axis in the order
    int R;
    float Rf;
    uint32_t cbias;  // kMagicBits - R
    int xdom32;      // neighbour domain along x: the column's 32-point block (else the chunk)
    int nseg[2][3][3];  // segments of pass k of level l, [plane 0 carried][l][k]
    int ord_id;         // index of the axis order (ord_axis)
    // the same values packed for single 16-byte loads in the fixed-geometry passes
    float4 q4[3];       // per level: e, 2e, 1/(2e), spline (0 or 1)
    int natural[3];     // per axis: natural cubic (else not-a-knot)
    uint4 k4;           // R, float(R) bits, cbias
    int dense_out;      // decompression: outliers exceed 1/64 of the points
};

// Dynamic shared memory of the tile kernels (layouts C_* and D_* above).
extern __shared__ __align__(128) unsigned char g_smem[];

// The kernels' copy of the per-call constants (one per CTA).  The pass functions
// read it by name, so its accesses stay shared-memory loads in out-of-line code.
__shared__ Levels g_lv;

__device__ __forceinline__ void load_levels(Levels &lv, const interp_header *h)
{
    for (int l = 0; l < 3; ++l) {
        lv.L[l].e = h->e[l];
        lv.L[l].twoe = h->twoe[l];
        lv.L[l].inv2e = h->inv2e[l];
        lv.spline[l] = h->cfg.level_kind[l];
        lv.cub[l] = cubic_coeffs(h->cfg.cubic_kind[l]);
        lv.order[l] = h->cfg.dim_order[l];
    }
    for (int k = 0; k < 3; ++k) lv.rank[lv.order[k]] = k;
    lv.ord_id = 2 * lv.order[0] + (lv.order[1] > lv.order[2] ? 1 : 0);
    lv.R = h->cfg.radius;
    lv.Rf = (float)lv.R;
    lv.cbias = kMagicBits - (uint32_t)lv.R;
    lv.xdom32 = h->cfg.domain_x == 32;
    lv.dense_out = h->n_outliers * 64ull > (unsigned long long)(h->dims[0] * h->dims[1] * h->dims[2]);
    for (int l = 0; l < 3; ++l) {
        lv.q4[l] = make_float4(lv.L[l].e, lv.L[l].twoe, lv.L[l].inv2e, lv.spline[l] ? 1.0f : 0.0f);
        lv.natural[l] = lv.cub[l].natural;
    }
    lv.k4 = make_uint4((uint32_t)lv.R, __float_as_uint(lv.Rf), lv.cbias, 0u);
    // segment counts of every pass (the same rule as run_pass), so that threads
    // without work in a pass leave it at once
    for (int carried = 0; carried < 2; ++carried)
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) {
                const int D = lv.order[k], S = 1 << l;
                const int U = axis_u(D), V = axis_v(D);
                const int nU = count_on(ext_of(U), lv.rank[U] < k ? S : 2 * S);
                const int nV = count_on(ext_of(V), lv.rank[V] < k ? S : 2 * S) - ((V == 0 && carried) ? 1 : 0);
                lv.nseg[carried][l][k] = nU * nV * chunks_of(D);
            }
}

// Slab c of an item covers planes [8c, 8c+8].  It writes the outputs of
// planes [8c, 8c+8] except: plane 8c when carried (the previous slab of the
// run wrote it as its plane 8), and plane 8c+8 when the run ends there and it
// is not the field's last plane (the next run starts with it).
__device__ __forceinline__ void slab_setup(Slab &s, const Field &f, int item, int c, int c_first, int c_last)
{
    const int col = item % f.cols;
    const int cx = col % f.cols_x, cy = col / f.cols_x;
    s.g0[0] = 8 * c;
    s.g0[1] = OY * cy;
    s.g0[2] = OX * cx;
    s.col = col;
    s.carried = c != c_first;
    s.own_lo = s.carried ? 1 : 0;
    const bool field_end = 8 * c + 8 == f.n[0] - 1;
    s.own_hi = (c != c_last || field_end) ? 8 : 7;
    s.lim[0] = min(s.own_hi, f.n[0] - 1 - s.g0[0]) + 1;
    s.lim[1] = min(OY, f.n[1] - s.g0[1]);
    s.lim[2] = min(OX, f.n[2] - s.g0[2]);
}

// ------------------------------------------------------------ passes
struct Sink {
    uint16_t *stage;       // compression: code staging
    const uint16_t *cbox;  // decompression: the slab's landed codes
    uint32_t *hist_s;      // compression: shared bins of codes 0 .. HIST_SMEM_BINS - 1
    uint32_t *hist_g;      // compression: global bins (codes beyond the shared ones), may be null
};

// Histogram of one owned point's code (Fig. 1, Sec. V-A).  The central code R
// is not counted: it is by far the most frequent one, and its bin is filled in
// after the tile kernel as N minus the other bins.  Code 0 (outliers) always
// lands in shared memory, which also tells the write-out whether a slab has
// outliers at all.
__device__ __forceinline__ void count_code(const Sink &sk, uint32_t code, uint32_t R, bool owned)
{
    if (owned && code != R) {
        if (code < (uint32_t)HIST_SMEM_BINS) atomicAdd(sk.hist_s + code, 1u);
        else if (sk.hist_g) atomicAdd(sk.hist_g + code, 1u);
    }
}

// INTERIOR: the slab's whole box lies inside the field and every chunk is
// full, so no line or chunk needs the field-edge checks.
template <bool COMPRESS, bool INTERIOR, int S, int D, bool XDOM = false>
__device__ __forceinline__ void run_pass(float *__restrict__ box, const Sink &sk, const Slab &sl, const Field &f,
                                         const Levels &lv, int k)
{
    constexpr int U = axis_u(D), V = axis_v(D);
    constexpr int EU = ext_of(U), EV = ext_of(V);
    constexpr int NC = chunks_of(D);
    constexpr int BD = bstride(D), BU = bstride(U), BV = bstride(V);
    constexpr int SD = sstride(D), SU = sstride(U), SV = sstride(V);
    constexpr int KD = lstride(D), KU = lstride(U), KV = lstride(V);
    constexpr int l = S == 1 ? 0 : (S == 2 ? 1 : 2);
    if ((int)threadIdx.x >= lv.nseg[sl.carried ? 1 : 0][l][k]) return;  // no segment for this thread

    // axes before D in the order sit on the s-grid, axes after it on the 2s-grid
    const bool ue = lv.rank[U] < k, ve = lv.rank[V] < k;
    const int stepU = ue ? S : 2 * S, stepV = ve ? S : 2 * S;
    const int nU = ue ? count_on(EU, S) : count_on(EU, 2 * S);
    const uint32_t mU = ue ? magic_of(count_on(EU, S)) : magic_of(count_on(EU, 2 * S));
    int nV = ve ? count_on(EV, S) : count_on(EV, 2 * S);
    int v0 = 0;
    uint32_t mV = ve ? magic_of(count_on(EV, S)) : magic_of(count_on(EV, 2 * S));
    if (V == 0 && sl.carried) {  // plane 0 is carried: skip its lines
        v0 = 1;
        nV -= 1;
        mV = ve ? magic_of(count_on(EV, S) - 1) : magic_of(count_on(EV, 2 * S) - 1);
    }
    const int nseg = nU * nV * NC;
    if ((int)threadIdx.x >= nseg) return;  // no segment for this thread in this pass

    const LevelQ Lq = lv.L[l];
    const bool spline = lv.spline[l] != 0;
    const Cubic cub = lv.cub[D];
    const float Rf = lv.Rf;
    const uint32_t cbias = lv.cbias;

    for (int w = threadIdx.x; w < nseg; w += NT) {
        // consecutive threads walk U first, then V, then the chunk along D
        const int q1 = fdiv(w, mU);
        const int iu = w - q1 * nU;
        const int cd = fdiv(q1, mV);
        const int iv = q1 - cd * nV + v0;
        const int u = iu * stepU, v = iv * stepV, dlo = 8 * cd;
        const int gd = sl.g0[D] + dlo;
        if (!INTERIOR && (sl.g0[U] + u >= f.n[U] || sl.g0[V] + v >= f.n[V] || gd + S > f.n[D] - 1)) continue;
        float *line = box + v * BV + u * BU + dlo * BD;
        const bool owned = u < own_of(U) && v < own_of(V);
        const bool counted = u < sl.lim[U] && v < sl.lim[V];  // owned and inside the field
        const int sbase = v * SV + u * SU + dlo * SD;
        const int cbase = v * KV + u * KU + dlo * KD;

        auto emit = [&](int o, float p) {
            if (COMPRESS) {
                const float x = line[o * BD];
                float xr;
                const uint32_t code = quantize(x, p, Lq, cbias, Rf, xr);
                line[o * BD] = xr;
                if (owned) sk.stage[sbase + o * SD] = (uint16_t)code;
                count_code(sk, code, (uint32_t)lv.R, counted);
            } else {
                // outliers (code 0) already hold their stored value in the box
                const uint32_t code = sk.cbox[cbase + o * KD];
                const float xq = p + code_to_q(code, cbias) * Lq.twoe;
                if (code) line[o * BD] = xq;
            }
        };

        const int hi = INTERIOR ? 8 : min(8, f.n[D] - 1 - gd);  // last offset of the (possibly truncated) chunk
        if (D == 2 && XDOM) {
            // x-extended domain (Sec. IV-C): neighbours anywhere in the column's
            // 32-point block, box x in [0, hiX]; the neighbour-count rule per point
            const int hiX = INTERIOR ? OX : min(OX, f.n[2] - 1 - sl.g0[2]);
#pragma unroll
            for (int o = S; o < 8; o += 2 * S) {
                if (o > hi) break;
                const int X = dlo + o;
                const bool has_m3 = X - 3 * S >= 0;
                const bool has_p1 = X + S <= hiX;
                const bool has_p3 = X + 3 * S <= hiX;
                const float m1 = line[(o - S) * BD];
                float p;
                if (!has_p1) {
                    p = m1;
                } else {
                    const float p1 = line[(o + S) * BD];
                    if (!spline) p = sp_linear(m1, p1);
                    else if (has_m3 && has_p3) p = sp_cubic(cub, line[(o - 3 * S) * BD], m1, p1, line[(o + 3 * S) * BD]);
                    else if (has_m3) p = sp_quad_left(line[(o - 3 * S) * BD], m1, p1);
                    else if (has_p3) p = sp_quad_right(m1, p1, line[(o + 3 * S) * BD]);
                    else p = sp_linear(m1, p1);
                }
                emit(o, p);
            }
        } else if (hi == 8) {
            if (S == 4) {
                emit(4, sp_linear(line[0], line[8 * BD]));
            } else if (S == 2) {
                const float k0 = line[0], k4 = line[4 * BD], k8 = line[8 * BD];
                if (spline) {
                    emit(2, sp_quad_right(k0, k4, k8));
                    emit(6, sp_quad_left(k0, k4, k8));
                } else {
                    emit(2, sp_linear(k0, k4));
                    emit(6, sp_linear(k4, k8));
                }
            } else {
                const float k0 = line[0], k2 = line[2 * BD], k4 = line[4 * BD], k6 = line[6 * BD],
                            k8 = line[8 * BD];
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
                const float m1 = line[(o - S) * BD];
                float p;
                if (!has_p1) {
                    p = m1;
                } else {
                    const float p1 = line[(o + S) * BD];
                    if (!spline) {
                        p = sp_linear(m1, p1);
                    } else if (has_m3 && has_p3) {
                        p = sp_cubic(cub, line[(o - 3 * S) * BD], m1, p1, line[(o + 3 * S) * BD]);
                    } else if (has_m3) {
                        p = sp_quad_left(line[(o - 3 * S) * BD], m1, p1);
                    } else if (has_p3) {
                        p = sp_quad_right(m1, p1, line[(o + 3 * S) * BD]);
                    } else {
                        p = sp_linear(m1, p1);
                    }
                }
                emit(o, p);
            }
        }
    }
}

template <bool COMPRESS, bool INTERIOR, int S, bool XDOM>
__device__ __forceinline__ void run_level(float *box, const Sink &sk, const Slab &sl, const Field &f,
                                          const Levels &lv)
{
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const int d = lv.order[k];
        if (d == 0) run_pass<COMPRESS, INTERIOR, S, 0>(box, sk, sl, f, lv, k);
        else if (d == 1) run_pass<COMPRESS, INTERIOR, S, 1>(box, sk, sl, f, lv, k);
        else run_pass<COMPRESS, INTERIOR, S, 2, XDOM>(box, sk, sl, f, lv, k);
        __syncthreads();
    }
}

template <bool COMPRESS, bool XDOM>
__device__ __forceinline__ void run_levels(float *box, const Sink &sk, const Slab &sl, const Field &f,
                                           const Levels &lv)
{
    const bool interior = sl.g0[0] + 8 <= f.n[0] - 1 && sl.g0[1] + OY <= f.n[1] - 1 && sl.g0[2] + OX <= f.n[2] - 1;
    if (interior) {
        run_level<COMPRESS, true, 4, XDOM>(box, sk, sl, f, lv);
        run_level<COMPRESS, true, 2, XDOM>(box, sk, sl, f, lv);
        run_level<COMPRESS, true, 1, XDOM>(box, sk, sl, f, lv);
    } else {
        run_level<COMPRESS, false, 4, XDOM>(box, sk, sl, f, lv);
        run_level<COMPRESS, false, 2, XDOM>(box, sk, sl, f, lv);
        run_level<COMPRESS, false, 1, XDOM>(box, sk, sl, f, lv);
    }
}


// ------------------------------------------------------------ passes with fixed geometry
// The default neighbour domain (the closed 8^3 chunk) with the axis order fixed at
// compile time: every pass's segment count, strides and line offsets are
// constants, so a thread decodes its segments with constant divisions and the
// loops unroll.  One instantiation per axis order (six) and per state of plane 0
// (carried or not); the kernel selects it once per slab.
//
// Axis orders are indexed 2*o0 + (o1 > o2): 012, 021, 102, 120, 201, 210.
__host__ __device__ constexpr int ord_axis(int ord, int k)
{
    // o0 = ord / 2; the two others in ascending order are (a, b); bit 0 swaps them
    return k == 0 ? ord / 2
                  : ((k == 1) == ((ord & 1) == 0) ? (ord / 2 == 0 ? 1 : 0) : (ord / 2 == 2 ? 1 : 2));
}
__host__ __device__ constexpr int ord_rank(int ord, int axis)
{
    return ord_axis(ord, 0) == axis ? 0 : (ord_axis(ord, 1) == axis ? 1 : 2);
}
static_assert(ord_axis(0, 1) == 1 && ord_axis(0, 2) == 2 && ord_axis(1, 1) == 2 && ord_axis(1, 2) == 1 &&
                  ord_axis(2, 0) == 1 && ord_axis(2, 1) == 0 && ord_axis(2, 2) == 2 && ord_axis(3, 1) == 2 &&
                  ord_axis(3, 2) == 0 && ord_axis(4, 1) == 0 && ord_axis(4, 2) == 1 && ord_axis(5, 1) == 1 &&
                  ord_axis(5, 2) == 0,
              "axis orders");

// Per-slab values of the fixed-geometry passes.
struct FastCtx {
    float *box;
    uint16_t *codes;  // code box: compression staging or decompression input (same layout)
    uint32_t *hist;   // compression: shared histogram bins (every code is below HIST_SMEM_BINS)
    int nfull[3];     // chunks along each axis that end inside the field (full chunks)
    int rem[3];       // last in-field offset along each axis, from the box origin
    int lim[3];       // owned in-field positions along each axis (Slab::lim)
};

// One point of a segment: compression quantizes and stages the code (the value
// stays in the box unless no later pass or slab reads it); decompression applies
// the stored code (code 0 = outlier, whose stored value is already in the box).
struct SegOut {
    uint32_t *hist;   // shared bins
    uint32_t *spare;  // this lane's spare word (updates that count nothing)
    uint32_t R;
    bool keep;       // the value is read again (compression)
    bool owned;      // the point's code is counted (compression)
};

template <bool COMPRESS>
__device__ __forceinline__ void seg_emit(float *L, uint16_t *C, int ob, int oc, float p, const LevelQ &Lq,
                                         uint32_t cbias, float Rf, const SegOut &so)
{
    if (COMPRESS) {
        float xr;
        const uint32_t code = quantize(L[ob], p, Lq, cbias, Rf, xr);
        if (so.keep) L[ob] = xr;
        C[oc] = (uint16_t)code;
        atomicAdd((so.owned && code != so.R) ? so.hist + code : so.spare, 1u);
    } else {
        const uint32_t code = C[oc];
        const float xq = p + code_to_q(code, cbias) * Lq.twoe;
        if (code) L[ob] = xq;
    }
}

// Decompression with the code already in a register.
__device__ __forceinline__ void seg_apply(float *L, int ob, float p, uint32_t code, const LevelQ &Lq, uint32_t cbias)
{
    const float xq = p + code_to_q(code, cbias) * Lq.twoe;
    if (code) L[ob] = xq;
}

// Prediction kinds of the fixed-geometry passes: linear only, or splines by
// neighbour count with the not-a-knot or the natural cubic.
enum { KIND_LINEAR = 0, KIND_NAK = 1, KIND_NATURAL = 2 };
template <int KIND>
__device__ __forceinline__ float cubic_of(float m3, float m1, float p1, float p3)
{
    return KIND == KIND_NATURAL ? sp_cubic_nat(m3, m1, p1, p3) : sp_cubic_nak(m3, m1, p1, p3);
}

// A segment of a full chunk: the fixed stencils of Fig. 3 (splines: cubic at
// offsets 3 and 5, quadratics at 1 and 7 for stride 1; quadratics at stride 2;
// stride 4 is always linear).
template <bool COMPRESS, int S, int BD, int KD, int KIND>
__device__ __forceinline__ void seg_full(float *L, uint16_t *C, const LevelQ &Lq, uint32_t cbias, float Rf,
                                         const SegOut &so)
{
    constexpr bool SPLINE = KIND != KIND_LINEAR;
    if (!COMPRESS && BD == 1 && KD == 1) {
        // decompression along x: the chunk row's 8 codes are one aligned 16-byte word
        // of the landed codes (rows of 80 bytes), so one load serves the segment
        const uint4 w = *reinterpret_cast<const uint4 *>(C);
        if (S == 4) {
            seg_apply(L, 4, sp_linear(L[0], L[8]), w.z & 0xffffu, Lq, cbias);
        } else if (S == 2) {
            const float k0 = L[0], k4 = L[4], k8 = L[8];
            seg_apply(L, 2, SPLINE ? sp_quad_right(k0, k4, k8) : sp_linear(k0, k4), w.y & 0xffffu, Lq, cbias);
            seg_apply(L, 6, SPLINE ? sp_quad_left(k0, k4, k8) : sp_linear(k4, k8), w.w & 0xffffu, Lq, cbias);
        } else {
            const float k0 = L[0], k2 = L[2], k4 = L[4], k6 = L[6], k8 = L[8];
            seg_apply(L, 1, SPLINE ? sp_quad_right(k0, k2, k4) : sp_linear(k0, k2), w.x >> 16, Lq, cbias);
            seg_apply(L, 3, SPLINE ? cubic_of<KIND>(k0, k2, k4, k6) : sp_linear(k2, k4), w.y >> 16, Lq, cbias);
            seg_apply(L, 5, SPLINE ? cubic_of<KIND>(k2, k4, k6, k8) : sp_linear(k4, k6), w.z >> 16, Lq, cbias);
            seg_apply(L, 7, SPLINE ? sp_quad_left(k4, k6, k8) : sp_linear(k6, k8), w.w >> 16, Lq, cbias);
        }
        return;
    }
    if (S == 4) {
        seg_emit<COMPRESS>(L, C, 4 * BD, 4 * KD, sp_linear(L[0], L[8 * BD]), Lq, cbias, Rf, so);
    } else if (S == 2) {
        const float k0 = L[0], k4 = L[4 * BD], k8 = L[8 * BD];
        seg_emit<COMPRESS>(L, C, 2 * BD, 2 * KD, SPLINE ? sp_quad_right(k0, k4, k8) : sp_linear(k0, k4), Lq, cbias,
                           Rf, so);
        seg_emit<COMPRESS>(L, C, 6 * BD, 6 * KD, SPLINE ? sp_quad_left(k0, k4, k8) : sp_linear(k4, k8), Lq, cbias,
                           Rf, so);
    } else {
        const float k0 = L[0], k2 = L[2 * BD], k4 = L[4 * BD], k6 = L[6 * BD], k8 = L[8 * BD];
        seg_emit<COMPRESS>(L, C, BD, KD, SPLINE ? sp_quad_right(k0, k2, k4) : sp_linear(k0, k2), Lq, cbias, Rf,
                           so);
        seg_emit<COMPRESS>(L, C, 3 * BD, 3 * KD, SPLINE ? cubic_of<KIND>(k0, k2, k4, k6) : sp_linear(k2, k4), Lq,
                           cbias, Rf, so);
        seg_emit<COMPRESS>(L, C, 5 * BD, 5 * KD, SPLINE ? cubic_of<KIND>(k2, k4, k6, k8) : sp_linear(k4, k6), Lq,
                           cbias, Rf, so);
        seg_emit<COMPRESS>(L, C, 7 * BD, 7 * KD, SPLINE ? sp_quad_left(k4, k6, k8) : sp_linear(k6, k8), Lq, cbias,
                           Rf, so);
    }
}

// A segment of a chunk cut by the field's far edge (last in-field offset hi < 8):
// the neighbour-count rule point by point (Sec. IV-B.1).
template <bool COMPRESS, int S, int BD, int KD>
__device__ __forceinline__ void seg_trunc(float *L, uint16_t *C, int hi, bool spline, const LevelQ &Lq,
                                          const Cubic &cub, uint32_t cbias, float Rf, const SegOut &so)
{
#pragma unroll
    for (int o = S; o < 8; o += 2 * S) {
        if (o > hi) break;
        const bool has_m3 = o - 3 * S >= 0;
        const bool has_p1 = o + S <= hi;
        const bool has_p3 = o + 3 * S <= hi;
        const float m1 = L[(o - S) * BD];
        float p;
        if (!has_p1) {
            p = m1;
        } else {
            const float p1 = L[(o + S) * BD];
            if (!spline) p = sp_linear(m1, p1);
            else if (has_m3 && has_p3) p = sp_cubic(cub, L[(o - 3 * S) * BD], m1, p1, L[(o + 3 * S) * BD]);
            else if (has_m3) p = sp_quad_left(L[(o - 3 * S) * BD], m1, p1);
            else if (has_p3) p = sp_quad_right(m1, p1, L[(o + 3 * S) * BD]);
            else p = sp_linear(m1, p1);
        }
        seg_emit<COMPRESS>(L, C, o * BD, o * KD, p, Lq, cbias, Rf, so);
    }
}

// Constants of one fixed-geometry pass.
struct PassK {
    LevelQ Lq;
    uint32_t cbias;
    float Rf;
    uint32_t R;
};

// Pass k of the level of stride S for axis order ORD.  Segments are numbered with
// U (the faster other axis) fastest, then V, then the chunk along D; thread t
// takes segments t, t + NT, ...  Threads without a segment skip the pass at once.
template <bool COMPRESS, int ORD, bool CARRIED, int S, int K, int KIND>
__device__ __forceinline__ void fast_pass(const FastCtx &c, const PassK &pk)
{
    constexpr bool SPLINE = KIND != KIND_LINEAR;
    constexpr int D = ord_axis(ORD, K);
    constexpr int U = axis_u(D), V = axis_v(D);
    constexpr int stepU = ord_rank(ORD, U) < K ? S : 2 * S;
    constexpr int stepV = ord_rank(ORD, V) < K ? S : 2 * S;
    constexpr int nU = count_on(ext_of(U), stepU);
    constexpr int v0 = (V == 0 && CARRIED) ? 1 : 0;  // plane 0 carried: its lines are done
    constexpr int nV = count_on(ext_of(V), stepV) - v0;
    constexpr int NC = chunks_of(D);
    constexpr int NSEG = nU * nV * NC;
    constexpr int BD = bstride(D), BU = bstride(U), BV = bstride(V);
    // codes: compression stages them in the code-box layout, decompression reads them as landed
    constexpr int KD = COMPRESS ? cstride(D) : lstride(D), KU = COMPRESS ? cstride(U) : lstride(U),
                  KV = COMPRESS ? cstride(V) : lstride(V);
    // after the last pass of compression only plane 8 (carried to the next slab) is read again
    constexpr bool LAST = COMPRESS && S == 1 && K == 2;
    const Cubic cub{KIND == KIND_NATURAL ? 1 : 0};  // truncated chunks choose per point
    SegOut so;
    so.hist = c.hist;
    so.spare = c.hist + HIST_SMEM_BINS + (threadIdx.x & 31);
    so.R = pk.R;
#pragma unroll 1
    for (int w = (int)threadIdx.x; w < NSEG; w += NT) {
        const int q1 = w / nU;
        const int iu = w - q1 * nU;
        const int cd = NC == 1 ? 0 : q1 / nV;
        const int iv = q1 - cd * nV + v0;
        const int u = iu * stepU, v = iv * stepV;
        float *L = c.box + v * BV + u * BU + 8 * cd * BD;
        uint16_t *C = c.codes + v * KV + u * KU + 8 * cd * KD;
        so.keep = !LAST || (D != 0 && v == 8);
        so.owned = u < c.lim[U] && v < c.lim[V];
        if (cd < c.nfull[D]) seg_full<COMPRESS, S, BD, KD, KIND>(L, C, pk.Lq, pk.cbias, pk.Rf, so);
        else seg_trunc<COMPRESS, S, BD, KD>(L, C, c.rem[D] - 8 * cd, SPLINE, pk.Lq, cub, pk.cbias, pk.Rf, so);
    }
}

template <bool COMPRESS, int ORD, bool CARRIED, int S, int K>
__device__ __forceinline__ void fast_pass_any(const FastCtx &c, const PassK &pk, bool spline)
{
    constexpr int D = ord_axis(ORD, K);
    constexpr int U = axis_u(D), V = axis_v(D);
    constexpr int nU = count_on(ext_of(U), ord_rank(ORD, U) < K ? S : 2 * S);
    constexpr int nV = count_on(ext_of(V), ord_rank(ORD, V) < K ? S : 2 * S) - ((V == 0 && CARRIED) ? 1 : 0);
    if ((int)threadIdx.x < nU * nV * chunks_of(D)) {
        // only stride 1 has four-neighbour (cubic) stencils inside a chunk
        if (!spline) fast_pass<COMPRESS, ORD, CARRIED, S, K, KIND_LINEAR>(c, pk);
        else if (S == 1 && g_lv.natural[D]) fast_pass<COMPRESS, ORD, CARRIED, S, K, KIND_NATURAL>(c, pk);
        else fast_pass<COMPRESS, ORD, CARRIED, S, K, KIND_NAK>(c, pk);
    }
    __syncthreads();
}

template <bool COMPRESS, int ORD, bool CARRIED, int S>
__device__ __forceinline__ void fast_level(const FastCtx &c, PassK pk)
{
    constexpr int l = S == 1 ? 0 : (S == 2 ? 1 : 2);
    const float4 q = g_lv.q4[l];
    pk.Lq = LevelQ{q.x, q.y, q.z};
    const bool spline = q.w != 0.0f;
    fast_pass_any<COMPRESS, ORD, CARRIED, S, 0>(c, pk, spline);
    fast_pass_any<COMPRESS, ORD, CARRIED, S, 1>(c, pk, spline);
    fast_pass_any<COMPRESS, ORD, CARRIED, S, 2>(c, pk, spline);
}

template <bool COMPRESS, int ORD>
__device__ __forceinline__ void fast_slab(const FastCtx &c, const PassK &pk, bool carried)
{
    if (carried) {
        fast_level<COMPRESS, ORD, true, 4>(c, pk);
        fast_level<COMPRESS, ORD, true, 2>(c, pk);
        fast_level<COMPRESS, ORD, true, 1>(c, pk);
    } else {
        fast_level<COMPRESS, ORD, false, 4>(c, pk);
        fast_level<COMPRESS, ORD, false, 2>(c, pk);
        fast_level<COMPRESS, ORD, false, 1>(c, pk);
    }
}

// The nine passes of a slab in the default neighbour domain, every order.
// The nine passes of a slab in the default neighbour domain, every order.
// rem: last in-field offset per axis from the box origin; lim: Slab::lim.
template <bool COMPRESS>
__device__ __forceinline__ void fast_levels(float *box, uint16_t *codes, uint32_t *hist, int rem0, int rem1,
                                            int rem2, int lim0, int lim1, int lim2, bool carried, const Levels &lv)
{
    FastCtx c;
    c.box = box;
    c.codes = codes;
    c.hist = hist;
    c.rem[0] = rem0;
    c.rem[1] = rem1;
    c.rem[2] = rem2;
    c.lim[0] = lim0;
    c.lim[1] = lim1;
    c.lim[2] = lim2;
#pragma unroll
    for (int a = 0; a < 3; ++a) c.nfull[a] = min(chunks_of(a), c.rem[a] / 8);
    const uint4 k = lv.k4;
    PassK pk;
    pk.R = k.x;
    pk.Rf = __uint_as_float(k.y);
    pk.cbias = k.z;
    switch (lv.ord_id) {
    case 0: fast_slab<COMPRESS, 0>(c, pk, carried); break;
    case 1: fast_slab<COMPRESS, 1>(c, pk, carried); break;
    case 2: fast_slab<COMPRESS, 2>(c, pk, carried); break;
    case 3: fast_slab<COMPRESS, 3>(c, pk, carried); break;
    case 4: fast_slab<COMPRESS, 4>(c, pk, carried); break;
    default: fast_slab<COMPRESS, 5>(c, pk, carried); break;
    }
}

// Pass dispatch.  The fixed-geometry passes serve the default neighbour domain;
// the x-extended domain (an option) and radii whose bins do not fit the shared
// histogram take the general passes.  Both are out-of-line functions, compiled
// once for every kernel that calls them (the call happens once per slab).
template <bool COMPRESS>
__device__ __noinline__ void passes_fast(int code_off, int rem0, int rem1, int rem2, int lim0, int lim1, int lim2,
                                         bool carried)
{
    // pointers derived from the shared-memory symbol, so that every access is a shared one
    float *box = reinterpret_cast<float *>(g_smem + (COMPRESS ? C_BOX : D_BOX));
    uint16_t *codes = reinterpret_cast<uint16_t *>(g_smem + code_off);
    uint32_t *hist = reinterpret_cast<uint32_t *>(g_smem + C_HIST);
    fast_levels<COMPRESS>(box, codes, hist, rem0, rem1, rem2, lim0, lim1, lim2, carried, g_lv);
}

template <bool COMPRESS>
__device__ __noinline__ void passes_general(const Slab sl, const Field f, uint32_t *hist_g)
{
    // shared-memory pointers derived from the symbol (not passed in), so that every box,
    // staging and bin access is a shared one and the slab's values stay in registers
    float *box = reinterpret_cast<float *>(g_smem + (COMPRESS ? C_BOX : D_BOX));
    const Sink sk{COMPRESS ? reinterpret_cast<uint16_t *>(g_smem + C_STAGE) : nullptr,
                  COMPRESS ? nullptr : reinterpret_cast<const uint16_t *>(g_smem + D_LAND),
                  COMPRESS ? reinterpret_cast<uint32_t *>(g_smem + C_HIST) : nullptr, hist_g};
    if (g_lv.xdom32) run_levels<COMPRESS, true>(box, sk, sl, f, g_lv);
    else run_levels<COMPRESS, false>(box, sk, sl, f, g_lv);
}

template <bool COMPRESS>
__device__ __forceinline__ void run_slab(float *box, const Sink &sk, const Slab &sl, const Field &f,
                                         const Levels &lv)
{
    // compression: the fixed-geometry passes keep every code's bin in shared memory
    const bool general = lv.xdom32 || (COMPRESS && 2 * lv.R > HIST_SMEM_BINS);
    if (general)
        passes_general<COMPRESS>(sl, f, sk.hist_g);  // box and sink at their fixed offsets
    else
        passes_fast<COMPRESS>((int)((COMPRESS ? reinterpret_cast<const unsigned char *>(sk.stage)
                                              : reinterpret_cast<const unsigned char *>(sk.cbox)) -
                                    g_smem),
                              f.n[0] - 1 - sl.g0[0], f.n[1] - 1 - sl.g0[1], f.n[2] - 1 - sl.g0[2], sl.lim[0],
                              sl.lim[1], sl.lim[2], sl.carried);
}

// ------------------------------------------------------------ work list
// Work items of all fields of a batch are numbered consecutively (field 0's
// items first).  A CTA takes items blockIdx.x, +gridDim.x, ...; an item is a
// run of up to f.run consecutive slabs of one column of one field.
template <typename FieldT>
struct BatchView {
    const FieldT *fld;
    int n, items;
};

struct Cursor {
    int item, fi, c, c_first, c_last;
};

template <bool MULTI, typename FieldT>
__device__ __forceinline__ bool cursor_start(Cursor &cu, const BatchView<FieldT> &b, int item)
{
    cu.item = item;
    if (item >= b.items) return false;
    int fi = 0;
    if (MULTI)
        while (fi + 1 < b.n && b.fld[fi + 1].item0 <= item) ++fi;
    cu.fi = fi;
    const Field &f = b.fld[fi].f;
    const int run_id = (item - b.fld[fi].item0) / f.cols;
    cu.c_first = run_id * f.run;
    cu.c_last = min(cu.c_first + f.run, f.slabs) - 1;
    cu.c = cu.c_first;
    return true;
}

template <bool MULTI, typename FieldT>
__device__ __forceinline__ bool cursor_next(Cursor &cu, const BatchView<FieldT> &b)
{
    if (cu.c < cu.c_last) {
        ++cu.c;
        return true;
    }
    return cursor_start<MULTI>(cu, b, cu.item + gridDim.x);
}

template <bool MULTI, typename FieldT>
__device__ __forceinline__ void slab_of(Slab &s, const Cursor &cu, const BatchView<FieldT> &b)
{
    const FieldT &F = b.fld[MULTI ? cu.fi : 0];
    slab_setup(s, F.f, cu.item - F.item0, cu.c, cu.c_first, cu.c_last);
}

// Bring the 9 x 17 x XP (or KP) input box of a slab into the landing buffer:
// one TMA box (thread 0; out-of-field elements are zero-filled), or, when the
// field's rows cannot be described by a tensor map, 4-byte cp.async copies
// of the in-field elements by all threads.
template <typename T, int P, int NPL, int Z0>
__device__ __forceinline__ void issue_land(T *land, const T *__restrict__ src, const CUtensorMap *map, bool use_tma,
                                           uint64_t *bar, const Field &f, const Slab &s)
{
    if (use_tma) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(T) * NPL * EY * P));
            tma_load_3d(land, map, s.g0[2], s.g0[1], s.g0[0] + Z0, bar);
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nzp = min(NPL, f.n[0] - s.g0[0] - Z0);
    const int nyr = min(EY, f.n[1] - s.g0[1]);
    const int nxc = min(EX, f.n[2] - s.g0[2]);
    for (int r = warp; r < nzp * EY; r += NWARP) {
        const int pz = r / EY, y = r % EY;
        if (y >= nyr) continue;
        const T *row = src + ((size_t)(s.g0[0] + Z0 + pz) * f.n[1] + s.g0[1] + y) * f.n[2] + s.g0[2];
        T *dst = land + r * P;
        if (sizeof(T) == 4) {
            if (lane < nxc) cp_async4(dst + lane, row + lane);
            if (lane == 0 && nxc > 32) cp_async4(dst + 32, row + 32);
        } else {
            if (lane < nxc) dst[lane] = row[lane];
            if (lane == 0 && nxc > 32) dst[32] = row[32];
        }
    }
    cp_async_commit();
}

// Wait for the landing transfer; false if it did not complete in time.
// The caller follows with a block barrier before reading the buffer.
__device__ __forceinline__ bool wait_land(bool use_tma, uint64_t *bar, uint32_t &phase)
{
    if (use_tma) {
        const bool ok = mbar_wait_bounded(bar, phase, kTmaPolls);
        phase ^= 1u;
        return ok;
    }
    cp_async_wait_all();
    return true;
}

// ------------------------------------------------------------ compression
struct CField {
    CompressArgs a;
    Field f;
    int item0;    // first batch item of this field
    int use_tma;  // input rows described by map[] (else cp.async path)
};

struct CBatch {
    CUtensorMap map[kMaxBatch];
    CField fld[kMaxBatch];
    int n, items;
};

// Per-field values of the compression write-out, re-read when the field changes.
struct CWrite {
    int R, Ay, Ax, WX;
    bool vec_codes;
    int code_store;
};

__device__ __forceinline__ CWrite cwrite_of(const CField &F)
{
    CWrite w;
    w.R = F.a.radius;
    w.Ay = (F.f.n[1] - 1) / 8 + 1;
    w.Ax = (F.f.n[2] - 1) / 8 + 1;
    w.WX = (F.f.n[2] + 31) / 32;
    w.vec_codes = F.a.vec_codes;
    w.code_store = F.a.code_store;
    return w;
}

// Add the CTA's histogram counts of one field to its global bins and clear them.
__device__ __forceinline__ void flush_hist(const CField &F, uint32_t *hist_s)
{
    __syncthreads();
    const int bins = min(2 * F.a.radius, HIST_SMEM_BINS);
    if (F.a.hist)
        for (int i = threadIdx.x; i < bins; i += NT) {
            const uint32_t h = hist_s[i];
            if (h) atomicAdd(&F.a.hist[i], h);
        }
    for (int i = threadIdx.x; i < HIST_SMEM_BINS; i += NT) hist_s[i] = 0u;
    __syncthreads();
}

// The owned planes of a slab whose rows all lie inside the field, with 16-byte
// aligned code rows and no outlier: staged codes -> global (8 codes per thread
// and store, three planes per step), anchors, and all-zero outlier-bitmap words.
static_assert(NT % 4 == 0 && (NT / 4) % OY == 0, "write-out steps cover whole planes");
__device__ __forceinline__ void write_slab_fast(const CField &F, const CWrite &cw, const Slab &sl, int rows,
                                                const uint16_t *stage, const float *box)
{
    const Field &f = F.f;
    constexpr int PSTEP = NT / 4 / OY;  // planes per step
    const int sub = threadIdx.x & 3;
    int r = threadIdx.x >> 2;
    const int y = r % OY;
    int pz = sl.own_lo + r / OY;
    const size_t plane = (size_t)f.n[1] * f.n[2];
    const uint16_t *sp = stage + pz * STAGE_PLANE + y * CP + 8 * sub;
    uint16_t *gp = F.a.codes + ((size_t)(sl.g0[0] + pz) * f.n[1] + sl.g0[1] + y) * f.n[2] + sl.g0[2] + 8 * sub;
    const bool anchor_row = (y & 7) == 0;
    for (; r < rows; r += NT / 4, pz += PSTEP, sp += PSTEP * STAGE_PLANE, gp += PSTEP * plane) {
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(sp);
        uint32_t w0 = s32[0];
        const uint32_t w1 = s32[1], w2 = s32[2], w3 = s32[3];
        if (anchor_row && (pz & 7) == 0) {  // anchor at x = 8*sub (Sec. IV-A): lossless, code R
            w0 = (w0 & 0xffff0000u) | (uint32_t)cw.R;
            const int gz = sl.g0[0] + pz, gy = sl.g0[1] + y, gx = sl.g0[2] + 8 * sub;
            F.a.anchors[((size_t)(gz / 8) * cw.Ay + gy / 8) * cw.Ax + gx / 8] = box[pz * PLANE + y * EX + 8 * sub];
        }
        *reinterpret_cast<uint4 *>(gp) = make_uint4(w0, w1, w2, w3);
    }
    // the slab's bitmap words are contiguous (16 per plane, tile-major layout)
    uint32_t *wb = F.a.bitmap + ((size_t)sl.col * f.n[0] + sl.g0[0] + sl.own_lo) * OY;
    if ((int)threadIdx.x < rows / 4) reinterpret_cast<uint4 *>(wb)[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
}

// Any other slab: codes stored as alignment allows, anchors, and the exact
// outlier-bitmap words with their block counts.  A warp takes 8 consecutive
// rows of one plane, 4 lanes x 8 codes per row.
__device__ __forceinline__ void write_slab_general(const CField &F, const CWrite &cw, const Slab &sl, int rows,
                                                   const uint16_t *stage, const float *box)
{
    const Field &f = F.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & 3;
    for (int base = warp * 8; base < rows; base += NWARP * 8) {
        const int row = base + (lane >> 2);
        const int pz = sl.own_lo + row / OY, y = row % OY;
        const int gz = sl.g0[0] + pz, gy = sl.g0[1] + y;
        const int gx = sl.g0[2] + 8 * sub;
        const bool rin = row < rows && gy < f.n[1];
        const int nvalid = rin ? min(8, f.n[2] - gx) : 0;  // in-field codes of this lane
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (row < rows) {
            const uint32_t *srow = reinterpret_cast<const uint32_t *>(stage + pz * STAGE_PLANE + y * CP + 8 * sub);
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = srow[j];
        }
        const size_t gi = ((size_t)gz * f.n[1] + gy) * f.n[2] + gx;
        if (nvalid > 0 && ((pz | y) & 7) == 0) {  // anchor at x = 8*sub (Sec. IV-A): lossless, code R
            w[0] = (w[0] & 0xffff0000u) | (uint32_t)cw.R;
            F.a.anchors[((size_t)(gz / 8) * cw.Ay + gy / 8) * cw.Ax + gx / 8] = box[pz * PLANE + y * EX + 8 * sub];
        }
        if (nvalid == 8 && cw.code_store == 8) {
            *reinterpret_cast<uint4 *>(F.a.codes + gi) = make_uint4(w[0], w[1], w[2], w[3]);
        } else if (nvalid == 8 && cw.code_store == 4) {
            reinterpret_cast<uint2 *>(F.a.codes + gi)[0] = make_uint2(w[0], w[1]);
            reinterpret_cast<uint2 *>(F.a.codes + gi)[1] = make_uint2(w[2], w[3]);
        } else if (nvalid == 8 && cw.code_store == 2) {
#pragma unroll
            for (int j = 0; j < 4; ++j) reinterpret_cast<uint32_t *>(F.a.codes + gi)[j] = w[j];
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < nvalid) F.a.codes[gi + j] = (uint16_t)(w[j >> 1] >> (16 * (j & 1)));
        }
        // outlier bits (code 0) of this lane's in-field codes
        uint32_t zmask = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            zmask |= (uint32_t)(j < nvalid && ((w[j >> 1] >> (16 * (j & 1))) & 0xffffu) == 0u) << j;
        // the 4 lanes of a row assemble its 32-bit outlier word
        uint32_t word = zmask << (8 * sub);
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        // tile-major bitmap: a slab's words are contiguous per plane
        if (sub == 0 && rin) F.a.bitmap[((size_t)sl.col * f.n[0] + gz) * OY + y] = word;
        // outlier counts per block of words (in ascending word order): the warp's 8 rows
        // nearly always fall into one block, so one atomic carries their sum
        const bool has = sub == 0 && rin && word != 0u;
        const uint32_t hm = __ballot_sync(0xffffffffu, has);
        if (hm) {
            const int64_t blk = (((int64_t)gz * f.n[1] + gy) * cw.WX + sl.g0[2] / 32) / BITMAP_BLOCK_WORDS;
            const int first = __ffs(hm) - 1;
            const long long b0 = __shfl_sync(0xffffffffu, (long long)blk, first);
            uint32_t c = has ? (uint32_t)__popc(word) : 0u;
            if (__all_sync(0xffffffffu, !has || blk == b0)) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
                if (lane == first) atomicAdd(&F.a.blockcnt[b0], c);
            } else if (has) {
                atomicAdd(&F.a.blockcnt[blk], c);
            }
        }
    }
}

// MULTI = false: a single field (index 0 everywhere, resolved at compile time).
template <bool MULTI>
__global__ void __launch_bounds__(NT, kCompressCtas) k_compress(const __grid_constant__ CBatch B)
{
    unsigned char *smem = g_smem;
    Levels &lv = g_lv;
    __shared__ int abort_flag;
    float *land = reinterpret_cast<float *>(smem + C_LAND);
    float *box = reinterpret_cast<float *>(smem + C_BOX);
    uint16_t *stage = reinterpret_cast<uint16_t *>(smem + C_STAGE);
    uint32_t *hist_s = reinterpret_cast<uint32_t *>(smem + C_HIST);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C_BAR);
    const BatchView<CField> bv{B.fld, B.n, B.items};

    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    for (int i = threadIdx.x; i < HIST_WORDS; i += NT) hist_s[i] = 0u;
    __syncthreads();

    uint32_t phase = 0;

    Cursor cu;
    if (!cursor_start<MULTI>(cu, bv, blockIdx.x)) return;
    Slab sl;
    slab_of<MULTI>(sl, cu, bv);
    int lv_field = -1;
    {
        const int fi = MULTI ? cu.fi : 0;
        issue_land<float, XP, XPL, 1>(land, B.fld[fi].a.x, &B.map[fi], B.fld[fi].use_tma, bar, B.fld[fi].f, sl);
    }
    for (;;) {
        const int fi = MULTI ? cu.fi : 0;
        const CField &F = B.fld[fi];
        const Field &f = F.f;
        const Sink sk{stage, nullptr, hist_s, F.a.hist};
        Cursor nx = cu;
        const bool has_next = cursor_next<MULTI>(nx, bv);
        Slab sn = sl;
        if (has_next) slab_of<MULTI>(sn, nx, bv);
        if (threadIdx.x == 0 && lv_field != fi) load_levels(lv, F.a.hdr);
        lv_field = fi;

        // ---- input: plane 0 carried, or loaded directly at a run's start; planes 1..8 landed
        if (!sl.carried) {
            const int nyr = min(EY, f.n[1] - sl.g0[1]), nxc = min(EX, f.n[2] - sl.g0[2]);
            const float *src = F.a.x + ((size_t)sl.g0[0] * f.n[1] + sl.g0[1]) * f.n[2] + sl.g0[2];
            for (int i = threadIdx.x; i < EY * EX; i += NT) {
                const int y = i / EX, xx = i - y * EX;
                if (y < nyr && xx < nxc) box[i] = __ldg(src + (size_t)y * f.n[2] + xx);
            }
        }
        if (!wait_land(F.use_tma, bar, phase)) abort_flag = 1;
        if (!F.use_tma) __syncthreads();  // cp.async copies of all threads visible
        for (int i = threadIdx.x; i < XPL * EY * 9; i += NT) {  // 9 groups of 4 floats per row (x 0..35)
            const int row = i / 9, q = i - 9 * row;
            const float4 v = *reinterpret_cast<const float4 *>(land + row * XP + 4 * q);
            float *d = box + (row + EY) * EX + 4 * q;  // landed row r is box row r + EY (plane + 1)
            d[0] = v.x;
            if (q < 8) {
                d[1] = v.y;
                d[2] = v.z;
                d[3] = v.w;
            }
        }
        __syncthreads();  // box and levels ready; the landing buffer now stages codes
        if (abort_flag) break;
        const uint32_t out0 = hist_s[0];  // outliers counted before this slab

        run_slab<true>(box, sk, sl, f, lv);  // ends with a barrier

        // ---- owned planes: codes, anchors, outlier-bitmap words
        const CWrite cw = cwrite_of(F);
        const int nzp = min(EZ, f.n[0] - sl.g0[0]);
        const int hi = min(sl.own_hi, nzp - 1);
        const int rows = (hi - sl.own_lo + 1) * OY;
        const bool outliers = hist_s[0] != out0;
        if (!outliers && cw.code_store == 8 && sl.g0[1] + OY <= f.n[1] && sl.g0[2] + OX <= f.n[2])
            write_slab_fast(F, cw, sl, rows, stage, box);
        else
            write_slab_general(F, cw, sl, rows, stage, box);
        // ---- next slab's input into the landing buffer (staged codes written out),
        // and plane 8 carried into plane 0 when the next slab continues this run
        __syncthreads();
        if (has_next) {
            const int nfi = MULTI ? nx.fi : 0;
            const CField &N = B.fld[nfi];
            issue_land<float, XP, XPL, 1>(land, N.a.x, &B.map[nfi], N.use_tma, bar, N.f, sn);
            if (nx.item == cu.item)
                for (int i = threadIdx.x; i < PLANE; i += NT) box[i] = box[8 * PLANE + i];
        }
        __syncthreads();  // box free for the next slab
        if (!has_next || (MULTI && nx.fi != cu.fi)) flush_hist(F, hist_s);  // field done
        if (!has_next) break;
        cu = nx;
        sl = sn;
    }
    if (abort_flag) {
        const int fi = MULTI ? cu.fi : 0;
        if (threadIdx.x == 0) {
            atomicOr(&B.fld[fi].a.hdr->status, INTERP_STATUS_TIMEOUT);
            // the transfer that did not arrive gets a second bounded wait before the
            // CTA's shared memory is released
            if (B.fld[fi].use_tma) mbar_wait_bounded(bar, phase ^ 1u, kTmaPolls);
        }
        flush_hist(B.fld[fi], hist_s);
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------- decompression
struct DField {
    DecompressArgs a;
    Field f;
    int item0;
    int use_tma;
};

struct DBatch {
    CUtensorMap map[kMaxBatch];
    DField fld[kMaxBatch];
    int n, items;
};

// The outliers (code 0) among a slab's landed codes: their values, which the
// scatter kernel put into xrec, go into the box.  A thread tests groups of 8
// codes (one 16-byte word) for a zero code.  DENSE (fields whose outliers exceed
// 1/64 of the points): a group with a zero fetches its 8 values with two 16-byte
// loads; otherwise each zero code fetches its own value, which keeps the loop
// that nearly never finds one short (measured faster on smooth fields, and
// slower by 30% on a field with 15% outliers).
template <bool DENSE>
__device__ __forceinline__ void land_outliers(float *box, const uint16_t *land, const DField &F, const Slab &sl)
{
    const Field &f = F.f;
    const int pz0 = sl.carried ? 1 : 0;
    const int nzp = min(EZ, f.n[0] - sl.g0[0]);
    const int nyr = min(EY, f.n[1] - sl.g0[1]);
    const int nxc = min(EX, f.n[2] - sl.g0[2]);
    const int nitem = (EZ - pz0) * EY * 5;  // 5 groups of 8 codes per row (x 0..39)
    // the landed rows are 5 groups each, so the groups of planes pz0.. are one flat run
    const uint4 *l4 = reinterpret_cast<const uint4 *>(land) + pz0 * EY * 5;
    for (int i = threadIdx.x; i < nitem; i += NT) {
        const uint4 v = l4[i];
        if (!(has_zero_half(v.x) | has_zero_half(v.y) | has_zero_half(v.z) | has_zero_half(v.w))) continue;
        const int row = pz0 * EY + i / 5, q = i % 5;
        if (q == 4 && !has_zero_half(v.x)) continue;  // the last group holds x = 32, 33 only
        const int pz = row / EY, y = row % EY;
        if (pz >= nzp || y >= nyr) continue;
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
        const int nj = min(8, min(nxc, EX) - 8 * q);  // in-field codes of the group
        if (DENSE) {
            const size_t g = ((size_t)(sl.g0[0] + pz) * f.n[1] + sl.g0[1] + y) * f.n[2] + sl.g0[2] + 8 * q;
            float *brow = box + row * EX + 8 * q;
            if (F.a.vec_xrec && nj == 8) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(F.a.xrec + g));
                const float4 b = __ldg(reinterpret_cast<const float4 *>(F.a.xrec + g) + 1);
                const float vals[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (((wv[j >> 1] >> (16 * (j & 1))) & 0xffffu) == 0u) brow[j] = vals[j];
            } else {
                for (int j = 0; j < nj; ++j)
                    if (((wv[j >> 1] >> (16 * (j & 1))) & 0xffffu) == 0u) brow[j] = __ldg(F.a.xrec + g + j);
            }
        } else {
            for (int j = 0; j < nj; ++j) {
                if (((wv[j >> 1] >> (16 * (j & 1))) & 0xffffu) == 0u) {
                    const size_t g =
                        ((size_t)(sl.g0[0] + pz) * f.n[1] + sl.g0[1] + y) * f.n[2] + sl.g0[2] + 8 * q + j;
                    box[row * EX + 8 * q + j] = __ldg(F.a.xrec + g);
                }
            }
        }
    }
}

// Decompression.  The codes of a slab land (TMA) in the landing buffer and the
// passes read them in place; the next slab's codes are issued as soon as the
// passes are done, so they land during the write-out, and the anchors of the
// next slab are fetched into registers before the current slab's passes.  One
// buffer (rather than two) lets six CTAs share an SM, whose extra warps hide
// the rest of the latency (measured faster than two buffers at five CTAs).
template <bool MULTI>
__global__ void __launch_bounds__(NT, kDecompressCtas) k_decompress(const __grid_constant__ DBatch B)
{
    unsigned char *smem = g_smem;
    Levels &lv = g_lv;
    __shared__ int abort_flag;
    float *box = reinterpret_cast<float *>(smem + D_BOX);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + D_BAR);
    const BatchView<DField> bv{B.fld, B.n, B.items};
    uint16_t *land = reinterpret_cast<uint16_t *>(smem + D_LAND);
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t phase = 0u;

    // anchors of a slab's planes 8 and (when not carried) 0: thread t < 2 * AYN * AXN holds one
    constexpr int AYN = OY / 8 + 1, AXN = OX / 8 + 1;  // anchor rows / columns of the box
    const int ai = threadIdx.x;
    const int a_z = ai / (AYN * AXN), a_y = (ai / AXN) % AYN, a_x = ai % AXN;
    const int a_off = (8 * a_z) * PLANE + (8 * a_y) * EX + 8 * a_x;
    auto anchor_fetch = [&](const DField &F, const Slab &s, float &v) {
        const Field &f = F.f;
        const int pz = 8 * a_z, y = 8 * a_y, x = 8 * a_x;
        const bool ok = ai < 2 * AYN * AXN && !(a_z == 0 && s.carried) && s.g0[0] + pz < f.n[0] &&
                        s.g0[1] + y < f.n[1] && s.g0[2] + x < f.n[2];
        if (ok) {
            const int Ay = (f.n[1] - 1) / 8 + 1, Ax = (f.n[2] - 1) / 8 + 1;
            v = __ldg(F.a.anchors + ((size_t)((s.g0[0] + pz) / 8) * Ay + (s.g0[1] + y) / 8) * Ax + (s.g0[2] + x) / 8);
        }
        return ok;
    };

    Cursor cu;
    if (!cursor_start<MULTI>(cu, bv, blockIdx.x)) return;
    Slab sl;
    slab_of<MULTI>(sl, cu, bv);
    // A single field whose outliers are all listed and number at most one per thread:
    // each thread keeps one outlier's coordinates, and a slab runs the outlier scan only
    // when one of them lies in its box (on smooth fields almost none does).
    bool few = false;
    int oz = -1, oy = 0, ox = 0;
    if (!MULTI) {
        const DField &F0 = B.fld[0];
        const unsigned long long nout = F0.a.hdr->n_outliers;
        few = F0.a.out_idx != nullptr && nout <= F0.a.out_capacity && nout <= (unsigned long long)NT;
        if (few && threadIdx.x < nout) {
            const uint32_t g = __ldg(F0.a.out_idx + threadIdx.x);
            const uint32_t plane = (uint32_t)F0.f.n[1] * (uint32_t)F0.f.n[2];
            oz = (int)(g / plane);
            const uint32_t r = g - (uint32_t)oz * plane;
            oy = (int)(r / (uint32_t)F0.f.n[2]);
            ox = (int)(r - (uint32_t)oy * (uint32_t)F0.f.n[2]);
        }
    }
    int lv_field = -1;
    float anc = 0.0f;
    bool anc_ok;
    {
        const int fi = MULTI ? cu.fi : 0;
        issue_land<uint16_t, KP, EZ, 0>(land, B.fld[fi].a.codes, &B.map[fi], B.fld[fi].use_tma, bar, B.fld[fi].f,
                                        sl);
        anc_ok = anchor_fetch(B.fld[fi], sl, anc);
    }
    for (;;) {
        const int fi = MULTI ? cu.fi : 0;
        const DField &F = B.fld[fi];
        const Field &f = F.f;
        Cursor nx = cu;
        const bool has_next = cursor_next<MULTI>(nx, bv);
        Slab sn = sl;
        if (has_next) slab_of<MULTI>(sn, nx, bv);
        if (threadIdx.x == 0 && lv_field != fi) load_levels(lv, F.a.hdr);
        lv_field = fi;

        // ---- this slab's codes
        if (!wait_land(F.use_tma, bar, phase)) abort_flag = 1;
        if (anc_ok) box[a_off] = anc;  // this slab's anchors, fetched a slab ago
        if (has_next) {
            const int nfi = MULTI ? nx.fi : 0;
            anc_ok = anchor_fetch(B.fld[nfi], sn, anc);
        }
        const bool mine = oz >= sl.g0[0] && oz < sl.g0[0] + EZ && oy >= sl.g0[1] && oy < sl.g0[1] + EY &&
                          ox >= sl.g0[2] && ox < sl.g0[2] + EX;
        // landed codes visible (cp.async: every thread's copies waited for), anchors and levels
        // too; and whether the slab's box may hold an outlier
        const bool scan = __syncthreads_or(!few || mine) != 0;
        // ---- outliers (code 0): their stored values, scattered into xrec, go into the box
        if (scan) {
            if (lv.dense_out) land_outliers<true>(box, land, F, sl);
            else land_outliers<false>(box, land, F, sl);
            __syncthreads();  // outlier values in the box
        }
        if (abort_flag) break;

        const Sink sk{nullptr, land, nullptr, nullptr};
        run_slab<false>(box, sk, sl, f, lv);  // ends with a barrier
        // ---- the codes are read: the next slab's land during the write-out
        if (has_next) {
            const int nfi = MULTI ? nx.fi : 0;
            const DField &N = B.fld[nfi];
            issue_land<uint16_t, KP, EZ, 0>(land, N.a.codes, &B.map[nfi], N.use_tma, bar, N.f, sn);
        }

        // ---- write the owned planes
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nzp = min(EZ, f.n[0] - sl.g0[0]);
        const int hi = min(sl.own_hi, nzp - 1);
        const int rows = (hi - sl.own_lo + 1) * OY;
        if (F.a.vec_xrec && sl.g0[1] + OY <= f.n[1] && sl.g0[2] + OX <= f.n[2]) {
            // whole rows, 16-byte aligned: 8 values per thread, three planes per step
            constexpr int PSTEP = NT / 4 / OY;
            const int sub4 = threadIdx.x & 3;
            int r = threadIdx.x >> 2;
            const int y = r % OY;
            const int pz = sl.own_lo + r / OY;
            const size_t plane = (size_t)f.n[1] * f.n[2];
            const float *sp = box + pz * PLANE + y * EX + 8 * sub4;
            float *gp = F.a.xrec + ((size_t)(sl.g0[0] + pz) * f.n[1] + sl.g0[1] + y) * f.n[2] + sl.g0[2] + 8 * sub4;
            for (; r < rows; r += NT / 4, sp += PSTEP * PLANE, gp += PSTEP * plane) {
                reinterpret_cast<float4 *>(gp)[0] = make_float4(sp[0], sp[1], sp[2], sp[3]);
                reinterpret_cast<float4 *>(gp)[1] = make_float4(sp[4], sp[5], sp[6], sp[7]);
            }
        } else {
            // 8 lanes x 4 values per row, 4 rows per warp
            const int sub = lane & 7;
            for (int base = warp * 4; base < rows; base += NWARP * 4) {
                const int row = base + (lane >> 3);
                const int pz = sl.own_lo + row / OY, y = row % OY;
                const int gz = sl.g0[0] + pz, gy = sl.g0[1] + y, gx = sl.g0[2] + 4 * sub;
                if (gy >= f.n[1] || gx >= f.n[2]) continue;
                const float *s4 = box + pz * PLANE + y * EX + 4 * sub;
                float *dst = F.a.xrec + ((size_t)gz * f.n[1] + gy) * f.n[2] + gx;
                if (F.a.vec_xrec && gx + 3 < f.n[2]) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(s4[0], s4[1], s4[2], s4[3]);
                } else {
                    for (int j = 0; j < 4 && gx + j < f.n[2]; ++j) dst[j] = s4[j];
                }
            }
        }
        __syncthreads();  // every thread is done reading the box
        if (!has_next) break;
        // ---- carry plane 8 into plane 0 of the next slab of the same run
        if (nx.item == cu.item) {
            for (int i = threadIdx.x; i < PLANE; i += NT) box[i] = box[8 * PLANE + i];
            __syncthreads();
        }
        cu = nx;
        sl = sn;
    }
    if (abort_flag && threadIdx.x == 0) {
        atomicOr(&const_cast<interp_header *>(B.fld[MULTI ? cu.fi : 0].a.hdr)->status, INTERP_STATUS_TIMEOUT);
        // the transfer that did not arrive (the only one issued: the next slab's is
        // issued after the passes) gets a second bounded wait before the CTA's shared
        // memory is released
        if (B.fld[MULTI ? cu.fi : 0].use_tma) mbar_wait_bounded(bar, phase ^ 1u, kTmaPolls);
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------ host side
constexpr int kMaxDevices = 64;
int compress_grid[2][kMaxDevices];  // [MULTI]
int decompress_grid[kMaxDevices], decompress_grid_multi[kMaxDevices];

// Opt in to the kernel's dynamic shared memory and size the persistent grid
// (resident CTAs per SM x SMs), once per device.
template <typename K>
cudaError_t prepare(K kernel, size_t smem, int *cache, int &grid)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && cache[dev] > 0) {
        grid = cache[dev];
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * sm_count();
    if (dev >= 0 && dev < kMaxDevices) cache[dev] = grid;
    return cudaSuccess;
}

Field field_of(Dims d)
{
    Field f;
    f.n[0] = d.nz;
    f.n[1] = d.ny;
    f.n[2] = d.nx;
    f.cols_x = (d.nx + OX - 1) / OX;
    f.cols = f.cols_x * ((d.ny + OY - 1) / OY);
    f.slabs = d.nz > 1 ? (d.nz - 1 + 7) / 8 : 1;
    f.run = f.slabs;
    f.items = f.cols;
    return f;
}

// Split the slabs of every column of every field into runs of one common
// length so that the busiest CTA of the persistent grid has the least work
// (each run start recomputes one plane); `forced` > 0 imposes the length.
void plan_runs(Field *fs, int n, int grid, int forced = 0)
{
    int max_slabs = 1;
    for (int i = 0; i < n; ++i) max_slabs = max(max_slabs, fs[i].slabs);
    int best_run = max_slabs;
    double best = 1e300;
    for (int run = 1; run <= max_slabs; ++run) {
        long long items = 0, work = 0;
        for (int i = 0; i < n; ++i) {
            items += (long long)fs[i].cols * ((fs[i].slabs + run - 1) / run);
            work += (long long)fs[i].cols * fs[i].slabs;
        }
        const long long per_cta = (items + grid - 1) / grid;
        // the busiest CTA's items, each the run length plus the cost of a run start
        // (plane 0 loaded and computed, the transfers not yet overlapped: about two
        // slabs), and the run length once more for the CTAs that idle while the last
        // items finish; fitted to 512^3 timings of runs 1 .. 64 (best: 8)
        const double cost = (double)per_cta * (run + 2.0) + 1.0 * run;
        (void)work;
        if (cost <= best + 1e-9) {  // ties: the longer run (fewer run starts)
            best = cost;
            best_run = run;
        }
    }
    if (forced > 0) best_run = forced;
    for (int i = 0; i < n; ++i) {
        fs[i].run = min(best_run, fs[i].slabs);
        fs[i].items = fs[i].cols * ((fs[i].slabs + fs[i].run - 1) / fs[i].run);
    }
}

}  // namespace

size_t bitmap_words_tiled(Dims d)
{
    const size_t cols = (size_t)((d.nx + OX - 1) / OX) * (size_t)((d.ny + OY - 1) / OY);
    return cols * (size_t)d.nz * OY;
}

// The grid of a persistent launch: the occupancy limit, or fewer CTAs per SM
// when the schedule asks for them.
int scheduled_grid(int grid, const TileSchedule *sched)
{
    if (sched && sched->ctas_per_sm > 0) grid = std::min(grid, sched->ctas_per_sm * sm_count());
    return std::max(grid, 1);
}

cudaError_t launch_compress_tiles(const CompressArgs *args, int n, cudaStream_t s, const TileSchedule *sched)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    int grid = 0;
    auto kernel = n > 1 ? k_compress<true> : k_compress<false>;
    cudaError_t e = prepare(kernel, kCompressSmem, compress_grid[n > 1 ? 1 : 0], grid);
    if (e != cudaSuccess) return e;
    grid = scheduled_grid(grid, sched);
    thread_local CBatch B;  // large parameter block, filled on the host
    std::memset(&B, 0, sizeof(B));
    Field fs[kMaxBatch];
    for (int i = 0; i < n; ++i) fs[i] = field_of(args[i].dims);
    plan_runs(fs, n, grid, sched ? sched->run : 0);
    int items = 0;
    for (int i = 0; i < n; ++i) {
        B.fld[i].a = args[i];
        B.fld[i].f = fs[i];
        B.fld[i].item0 = items;
        items += fs[i].items;
        const uint32_t box[3] = {XP, EY, XPL};  // planes 1..8 of a slab: must match issue_land<float, XP, XPL, 1>
        B.fld[i].use_tma =
            encode_tensor_map_3d(&B.map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, args[i].x, args[i].dims, box) ? 1 : 0;
    }
    B.n = n;
    B.items = items;
    if (items < grid) grid = items;
    kernel<<<grid, NT, kCompressSmem, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_decompress_tiles(const DecompressArgs *args, int n, cudaStream_t s, const TileSchedule *sched)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    int grid = 0;
    cudaError_t e = n > 1 ? prepare(k_decompress<true>, kDecompressSmem, decompress_grid_multi, grid)
                          : prepare(k_decompress<false>, kDecompressSmem, decompress_grid, grid);
    if (e != cudaSuccess) return e;
    grid = scheduled_grid(grid, sched);
    thread_local DBatch B;
    std::memset(&B, 0, sizeof(B));
    Field fs[kMaxBatch];
    for (int i = 0; i < n; ++i) fs[i] = field_of(args[i].dims);
    plan_runs(fs, n, grid, sched ? sched->run : 0);
    int items = 0;
    for (int i = 0; i < n; ++i) {
        B.fld[i].a = args[i];
        B.fld[i].f = fs[i];
        B.fld[i].item0 = items;
        items += fs[i].items;
        const uint32_t box[3] = {KP, EY, EZ};
        B.fld[i].use_tma =
            encode_tensor_map_3d(&B.map[i], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, args[i].codes, args[i].dims, box) ? 1
                                                                                                                   : 0;
    }
    B.n = n;
    B.items = items;
    if (items < grid) grid = items;
    if (n > 1) k_decompress<true><<<grid, NT, kDecompressSmem, s>>>(B);
    else k_decompress<false><<<grid, NT, kDecompressSmem, s>>>(B);
    return cudaGetLastError();
}

// ------------------------------------------------------------ tensor maps
bool encode_tensor_map_3d(CUtensorMap *map, CUtensorMapDataType dtype, size_t elem, const void *base, Dims d,
                          const uint32_t box[3])
{
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        looked_up = true;
    }
    if (!fn) return false;
    const size_t row_bytes = elem * (size_t)d.nx;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || row_bytes % 16 != 0) return false;
    const cuuint64_t gdim[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t gstride[2] = {(cuuint64_t)row_bytes, (cuuint64_t)row_bytes * (cuuint64_t)d.ny};
    const cuuint32_t bdim[3] = {box[0], box[1], box[2]};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult r = fn(map, dtype, 3, const_cast<void *>(base), gdim, gstride, bdim, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace gi
