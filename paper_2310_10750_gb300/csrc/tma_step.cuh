// Persistent streaming step kernel with TMA tile loads.
//
// Fields between steps live in library scratch with a periodic ghost frame of width
// G = R4 (R rounded up to a multiple of 4): a padded n+2G square per sample whose frame
// holds the periodic images of the opposite edges.  A tile plus its R-wide halo is then
// one contiguous box of the padded array, fetched by one cp.async.bulk.tensor (TMA)
// copy without any index wrapping.  Each CTA loops over (sample, tile) items with two
// shared-memory stages: the TMA copy of the next item is in flight while the current one
// is computed.  Every output is written to its interior position and, near an edge, to
// its ghost images, so the next step's tiles find their halos in place.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "step_kernels.cuh"

namespace mfmc {

struct TmaArgs {
    float *dst;            // padded destination (nullptr: no field output)
    float *dst_plain;      // unpadded destination (last step with a final field), or nullptr
    const StepCoef *coef;
    double *partials;      // [ns][tiles], written at the last step
    int *status;           // set to 1 when a bounded wait gives up
    const int *steps_ps;   // per-sample step counts (serving), or nullptr: every sample runs `step`
    int step;              // 1-based index of this step
    int n, P, tiles_x, tiles, total, last;
    int periodic;          // 1: periodic frame (outputs also stored as ghost images); 0: the frame
                           // is a fixed collar and only interior outputs are stored
    const float *wsq;      // weighted sums (ALGO 3): [(R + 1) * (R + 1)] weights by (|dy|, |dx|), zero
                           // outside the disc; nullptr for the prefix forms
};

// A sample takes part in step `a.step` while a.step <= its own step count.
__device__ __forceinline__ bool item_active(const TmaArgs &a, int item) {
    return a.steps_ps == nullptr || a.step <= a.steps_ps[item / a.tiles];
}

__device__ __forceinline__ int next_active(const TmaArgs &a, int item, int stride) {
    while (item < a.total && !item_active(a, item)) item += stride;
    return item;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

template <int R, int RY, int TXT, int TYT, int STAGES = 2>
struct TmaCfg {
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int TX = 4 * TXT, TY = RY * TYT;
    static constexpr int SW = TX + 2 * R4, SH = TY + 2 * R;
    static constexpr int STAGE_FLOATS = ((SW * SH + 255) / 256) * 256;  // 1 KB aligned stages
    static constexpr size_t SMEM = STAGES * (size_t)STAGE_FLOATS * sizeof(float) + 1024;
    static constexpr uint32_t BOX_BYTES = (uint32_t)SW * SH * sizeof(float);
};

constexpr long long kWaitLimit = 1ll << 24;

// Store one float4 at padded (row, col) of a field with row pitch P when both are >= 0
// (a ghost image that exists).
__device__ __forceinline__ void put_ghost(float *d, int P, int row, int col, float4 val) {
    if (row >= 0 && col >= 0) *reinterpret_cast<float4 *>(d + (size_t)row * P + col) = val;
}

// Where one thread's outputs of an item go: the sample's padded destination (with the
// periodic ghost images) or its unpadded destination, and the thread's ghost column.
struct TmaRowCtx {
    float *d;       // padded destination of the sample, or nullptr
    float *dp;      // unpadded destination of the sample, or nullptr
    bool framed;    // the thread's block touches the frame (periodic lattice only)
    bool one_image; // n >= 2G: a row or column has at most one ghost image
    int cxg;        // padded column of the block's ghost image, or -1
};

// Flags of an output row's epilogue: which stores it makes and whether it adds to the OoI.
enum : unsigned { kRowPlain = 1u, kRowPadded = 2u, kRowFramed = 4u, kRowOneImage = 8u, kRowLast = 16u };

__host__ __device__ __forceinline__ unsigned tma_row_flags(const TmaRowCtx &c, bool last) {
    return (c.dp ? kRowPlain : 0u) | (!c.dp && c.d ? kRowPadded : 0u) | (c.framed ? kRowFramed : 0u) |
           (c.one_image ? kRowOneImage : 0u) | (last ? kRowLast : 0u);
}

// The value of x through an instruction the compiler cannot move: branches on flags that are
// fixed for a whole item then stay inside the unrolled row loop instead of making the compiler
// copy the loop once per flag combination (which multiplied the code and stalled instruction
// fetch).
__device__ __forceinline__ unsigned opaque_u32(unsigned x) {
    unsigned y;
    asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

template <int R>
__device__ __forceinline__ TmaRowCtx tma_row_ctx(const TmaArgs &a, int sample, int xg, int yg, int ry) {
    constexpr int RX = 4, G = (R + 3) & ~3;
    const int n = a.n;
    TmaRowCtx c;
    c.dp = a.dst_plain ? a.dst_plain + (size_t)sample * n * n : nullptr;
    c.d = (!a.dst_plain && a.dst) ? a.dst + (size_t)sample * a.P * a.P : nullptr;
    c.framed = a.periodic && (xg < G || xg + RX > n - G || yg < G || yg + ry > n - G);
    c.one_image = n >= 2 * G;
    c.cxg = xg < G ? G + xg + n : (xg >= n - G ? G + xg - n : -1);
    return c;
}

// The update and projection of one output row of a thread (four columns at lattice (y, x))
// from its disc sums (s01, s23) and centre values uc, the store of the row (and, on the
// periodic lattice, of its ghost images); adds the row's FP64 sum to `part` when `last`
// (only then: FP64 arithmetic runs at a small fraction of the FP32 rate on this part).
// Packed FP32 pairs round exactly like the scalar operations they replace:
//   sd = fma(-c0, u, S),  v = u + fma(c1, sd, c2 u),  u_new = min(1, max(-1, v)).
// PART = false: no OoI partial (the caller reduces the final field separately); GENERAL =
// false: the field is at least twice the frame width, so only the single-image ghost path is
// built; OPAQUE: the flags pass through opaque_u32 (for callers whose row loop the compiler
// would otherwise copy per flag combination).
template <int R, bool PART = true, bool GENERAL = true, bool OPAQUE = false>
__device__ __forceinline__ void tma_emit_row(const TmaArgs &a, const TmaRowCtx &c, const StepCoef &cf,
                                             float4 uc, float2 s01, float2 s23, int y, int x, bool last_in,
                                             double &part) {
    constexpr int G = (R + 3) & ~3;
    const int n = a.n;
    const unsigned fl = OPAQUE ? opaque_u32(tma_row_flags(c, last_in)) : tma_row_flags(c, last_in);
    const bool last = fl & kRowLast;
    const float2 nc0 = make_float2(-cf.c0, -cf.c0), c1 = make_float2(cf.c1, cf.c1),
                 c2 = make_float2(cf.c2, cf.c2);
    const float2 u01 = make_float2(uc.x, uc.y), u23 = make_float2(uc.z, uc.w);
    const float2 v01 = __fadd2_rn(u01, __ffma2_rn(c1, __ffma2_rn(nc0, u01, s01), __fmul2_rn(c2, u01)));
    const float2 v23 = __fadd2_rn(u23, __ffma2_rn(c1, __ffma2_rn(nc0, u23, s23), __fmul2_rn(c2, u23)));
    const float4 val = make_float4(fminf(1.f, fmaxf(-1.f, v01.x)), fminf(1.f, fmaxf(-1.f, v01.y)),
                                   fminf(1.f, fmaxf(-1.f, v23.x)), fminf(1.f, fmaxf(-1.f, v23.y)));
    if (y >= n || x >= n) return;
    if (fl & kRowPlain) {
        *reinterpret_cast<float4 *>(c.dp + (size_t)y * n + x) = val;
    } else if (fl & kRowPadded) {
        float *d = c.d;
        *reinterpret_cast<float4 *>(d + (size_t)(G + y) * a.P + G + x) = val;
        if ((fl & (kRowFramed | kRowOneImage)) == (kRowFramed | kRowOneImage)) {
            const int ry = y < G ? G + y + n : (y >= n - G ? G + y - n : -1);
            put_ghost(d, a.P, G + y, c.cxg, val);
            if (ry >= 0) {
                *reinterpret_cast<float4 *>(d + (size_t)ry * a.P + G + x) = val;
                put_ghost(d, a.P, ry, c.cxg, val);
            }
        } else if (GENERAL && (fl & kRowFramed)) {
            // ghost images at rows G + y +- n and columns G + x +- n inside the frame
            const int ra = y < G ? G + y + n : -1, rb = y >= n - G ? G + y - n : -1;
            const int ca = x < G ? G + x + n : -1, cb = x >= n - G ? G + x - n : -1;
            put_ghost(d, a.P, G + y, ca, val);
            put_ghost(d, a.P, G + y, cb, val);
            put_ghost(d, a.P, ra, G + x, val);
            put_ghost(d, a.P, ra, ca, val);
            put_ghost(d, a.P, ra, cb, val);
            put_ghost(d, a.P, rb, G + x, val);
            put_ghost(d, a.P, rb, ca, val);
            put_ghost(d, a.P, rb, cb, val);
        }
    }
    if (PART && last) part += ((double)val.x + (double)val.y) + ((double)val.z + (double)val.w);
}

// The FP64 OoI partial of a tile: the block's fixed-order sum of its threads' row sums.
template <int NT>
__device__ __forceinline__ void tma_tile_partial(const TmaArgs &a, int sample, int tile, double part, double *red) {
    const double t = block_sum_fixed<NT>(part, red);
    if (threadIdx.x == 0) a.partials[(size_t)sample * a.tiles + tile] = t;
}

// One staged row as a thread's four output columns read it: the window v of RX + 2 R4 values
// (staged columns ox .. ox + RX + 2 R4 - 1, output column i at window index R4 + i), and its
// centre sums p over the window's columns k = 0 .. RX + 2R - 1 (window index R4 - R + k), two
// independent chains from the middle M = RX / 2 + R:
//   p[k] = sum_{M <= m < k} for k > M,   p[k] = sum_{k <= m < M} for k < M,   p[M] = 0.
template <int R>
struct RowWin {
    static constexpr int RX = 4, R4 = (R + 3) & ~3, WIN = RX + 2 * R4, NP = RX + 2 * R + 1, M = RX / 2 + R;
    float v[WIN];
    float p[NP];
};

// The centre sums p of a window whose values v are loaded.
template <int R>
__device__ __forceinline__ void row_prefix(RowWin<R> &w) {
    using W = RowWin<R>;
    constexpr int M = W::M, o = W::R4 - R;
    w.p[M] = 0.f;
    w.p[M + 1] = w.v[o + M];
    w.p[M - 1] = w.v[o + M - 1];
#pragma unroll
    for (int q = 1; q < M; ++q) {
        w.p[M + 1 + q] = w.p[M + q] + w.v[o + M + q];
        w.p[M - 1 - q] = w.p[M - q] + w.v[o + M - 1 - q];
    }
}

template <int R>
__device__ __forceinline__ void row_window(const float *rowp, RowWin<R> &w) {
    using W = RowWin<R>;
    const float4 *r4 = reinterpret_cast<const float4 *>(rowp);
#pragma unroll
    for (int q = 0; q < W::WIN / 4; ++q) {
        const float4 x = r4[q];
        w.v[4 * q + 0] = x.x;
        w.v[4 * q + 1] = x.y;
        w.v[4 * q + 2] = x.z;
        w.v[4 * q + 3] = x.w;
    }
    row_prefix<R>(w);
}

// The four row-segment sums of half-width HW centred on the thread's output columns i = 0..3:
// window columns [i + R - HW, i + R + HW + 1) from the centre sums (a segment right of, left of
// or across the middle is p[e] - p[b], p[b] - p[e] or p[e] + p[b]); HW = 0 is the centre value.
template <int R, int HW>
__device__ __forceinline__ void class_sums(const RowWin<R> &w, float (&h)[4]) {
    constexpr int M = RowWin<R>::M, R4 = RowWin<R>::R4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int b = i + R - HW, e = i + R + HW + 1;
        if constexpr (HW == 0)
            h[i] = w.v[R4 + i];
        else
            h[i] = b >= M ? w.p[e] - w.p[b] : (e <= M ? w.p[b] - w.p[e] : w.p[e] + w.p[b]);
    }
}

// Static plan of the constant-kernel tile sums: which output rows j of a 4 x RY block the
// staged row r serves, and through which half-width class (dy = r - R - j).
template <int R, int RY>
struct TilePlan {
    static constexpr DiscClasses<R> cls{};
    __host__ __device__ static constexpr bool serves(int r, int j, int c) {
        const int dy = r - R - j, ady = dy < 0 ? -dy : dy;
        return ady <= R && cls.of[ady] == c;
    }
    __host__ __device__ static constexpr bool used(int r, int c) {
        for (int j = 0; j < RY; ++j)
            if (serves(r, j, c)) return true;
        return false;
    }
};

// Accumulators of a thread's block: packed pairs (ALGO 1) or compensated scalars (ALGO 2).
template <int RY, int ALGO>
struct TileAcc {
    float2 acc[RY][2];
    float kacc[ALGO == 2 ? RY : 1][4], cmp[ALGO == 2 ? RY : 1][4];
};

template <int R, int RY, int ALGO, int r, int c, int j>
__device__ __forceinline__ void tile_add(TileAcc<RY, ALGO> &t, const float (&h)[4]) {
    if constexpr (TilePlan<R, RY>::serves(r, j, c)) {
        constexpr bool first = r == j;  // dy = -R: the output row's first staged row
        if constexpr (ALGO != 2) {
            const float2 h01 = make_float2(h[0], h[1]), h23 = make_float2(h[2], h[3]);
            if constexpr (first) {
                t.acc[j][0] = h01;
                t.acc[j][1] = h23;
            } else {
                t.acc[j][0] = __fadd2_rn(t.acc[j][0], h01);
                t.acc[j][1] = __fadd2_rn(t.acc[j][1], h23);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if constexpr (first) {
                    t.kacc[j][i] = h[i];
                    t.cmp[j][i] = 0.f;
                } else {
                    const float yk = h[i] - t.cmp[j][i];
                    const float s = t.kacc[j][i] + yk;
                    t.cmp[j][i] = (s - t.kacc[j][i]) - yk;
                    t.kacc[j][i] = s;
                }
            }
        }
    }
}

// The four segment sums of class c in staged row r (once per row), added to every output
// row the class serves.
template <int R, int RY, int ALGO, int r, int c, int... J>
__device__ __forceinline__ void tile_class(TileAcc<RY, ALGO> &t, const RowWin<R> &win,
                                           std::integer_sequence<int, J...>) {
    if constexpr (TilePlan<R, RY>::used(r, c)) {
        float h[4];
        class_sums<R, TilePlan<R, RY>::cls.width[c]>(win, h);
        (tile_add<R, RY, ALGO, r, c, J>(t, h), ...);
    }
}

// Per-item state of a thread for the output rows it emits.
struct TileEmit {
    const float *s;
    const TmaArgs *a;
    TmaRowCtx ctx;
    StepCoef cf;
    int ox, oy, x0, y0;
    bool last;
    double part;
};

// Staged row r: its window, its prefix sums, the class sums; then, once r >= 2R, the update
// and store of output row r - 2R, whose disc is complete.
template <int R, int RY, int TXT, int ALGO, int r, int... C>
__device__ __forceinline__ void tile_row(TileAcc<RY, ALGO> &t, TileEmit &e, std::integer_sequence<int, C...>) {
    constexpr int RX = 4, R4 = (R + 3) & ~3, SW = 4 * TXT + 2 * R4;
    RowWin<R> win;
    row_window<R>(e.s + (e.oy + r) * SW + e.ox, win);
    (tile_class<R, RY, ALGO, r, C>(t, win, std::make_integer_sequence<int, RY>{}), ...);
    if constexpr (r >= 2 * R) {
        constexpr int j = r - 2 * R;
        const float4 uc = *reinterpret_cast<const float4 *>(e.s + (e.oy + j + R) * SW + e.ox + R4);
        float2 s01, s23;
        if constexpr (ALGO != 2) {
            s01 = t.acc[j][0];
            s23 = t.acc[j][1];
        } else {
            s01 = make_float2(t.kacc[j][0], t.kacc[j][1]);
            s23 = make_float2(t.kacc[j][2], t.kacc[j][3]);
        }
        tma_emit_row<R>(*e.a, e.ctx, e.cf, uc, s01, s23, e.y0 + e.oy + j, e.x0 + e.ox, e.last, e.part);
    }
}

template <int R, int RY, int TXT, int ALGO, int... Rows>
__device__ __forceinline__ void tile_rows(TileAcc<RY, ALGO> &t, TileEmit &e, std::integer_sequence<int, Rows...>) {
    (tile_row<R, RY, TXT, ALGO, Rows>(t, e, std::make_integer_sequence<int, TilePlan<R, RY>::cls.count>{}), ...);
}

// One tile item of the constant kernel: disc sums from the staged tile `s` (tile + halo, row
// pitch SW), the update and projection, stores of the outputs (and ghost images), and the
// FP64 partial of the OoI when `last`.  Shared by the single-fidelity and the mixed-fidelity
// kernels.
//
// A thread owns a 4 x RY block of outputs and walks the RY + 2R staged rows that its block
// reads.  From each row's window it forms an in-register prefix sum p; the segment sum of
// half-width w centred on output column i is p[i + R + w + 1] - p[i + R - w] (for w = 0 the
// centre value itself).  Rows of one half-width class serve several output rows of the block,
// so each class's four segment sums are formed once per staged row and added to every output
// row that class serves (in packed FP32 pairs for ALGO 1; compensated scalar sums for ALGO 2).
// An output row is complete after staged row j + 2R: its update and store follow at once, so
// at most 2R + 1 output rows hold accumulators at any time.  The row, class and output-row
// structure is generated at compile time, so every accumulator index is static.
template <int R, int RY, int TXT, int TYT>
__device__ __forceinline__ void tma_tile_epilogue(const float *s, const TmaArgs &a, int sample, int tile, int x0,
                                                  int y0, bool last, double *red, const StepCoef &cf,
                                                  const float (&acc)[RY][4]);

// Horizons above 16 (up to 32 half-width classes and 2R + RY staged rows): one segment sum per
// (staged row, output row) from the same row prefix, accumulated in that row order, and the
// updates after the last row (the class plan would unroll into too much code).
template <int R, int RY, int TXT, int TYT, int ALGO>
__device__ __forceinline__ void tma_tile_compute_seg(const float *s, const TmaArgs &a, int sample, int tile, int x0,
                                                     int y0, bool last, double *red) {
    constexpr int RX = 4, R4 = (R + 3) & ~3, SW = 4 * TXT + 2 * R4, WIN = RX + 2 * R4;
    constexpr DiscRows<R> disc{};
    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT, ox = tx * RX, oy = ty * RY;
    const StepCoef cf = a.coef[sample];
    float acc[RY][RX];
    float cmp[ALGO == 2 ? RY : 1][RX];
#pragma unroll
    for (int j = 0; j < RY; ++j)
#pragma unroll
        for (int i = 0; i < RX; ++i) {
            acc[j][i] = 0.f;
            cmp[ALGO == 2 ? j : 0][i] = 0.f;
        }
#pragma unroll
    for (int r = 0; r < RY + 2 * R; ++r) {
        const float4 *rowp = reinterpret_cast<const float4 *>(s + (oy + r) * SW + ox);
        float v[WIN];
#pragma unroll
        for (int q = 0; q < WIN / 4; ++q) {
            const float4 t = rowp[q];
            v[4 * q + 0] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
        float p[RX + 2 * R + 1];
        p[0] = 0.f;
#pragma unroll
        for (int q = 0; q < RX + 2 * R; ++q) p[q + 1] = p[q] + v[R4 - R + q];
#pragma unroll
        for (int j = 0; j < RY; ++j) {
            const int dy = r - R - j;
            if (dy >= -R && dy <= R) {
                const int w = disc.w[dy < 0 ? -dy : dy];
#pragma unroll
                for (int i = 0; i < RX; ++i) {
                    const float h = p[i + R + w + 1] - p[i + R - w];
                    if (ALGO != 2) {
                        acc[j][i] += h;
                    } else {
                        const float y = h - cmp[ALGO == 2 ? j : 0][i];
                        const float t = acc[j][i] + y;
                        cmp[ALGO == 2 ? j : 0][i] = (t - acc[j][i]) - y;
                        acc[j][i] = t;
                    }
                }
            }
        }
    }
    tma_tile_epilogue<R, RY, TXT, TYT>(s, a, sample, tile, x0, y0, last, red, cf, acc);
}

template <int R, int RY, int TXT, int TYT, int ALGO>
__device__ __forceinline__ void tma_tile_compute(const float *s, const TmaArgs &a, int sample, int tile, int x0,
                                                 int y0, bool last, double *red) {
    if constexpr (R > 16) {
        tma_tile_compute_seg<R, RY, TXT, TYT, ALGO>(s, a, sample, tile, x0, y0, last, red);
    } else {
        constexpr int RX = 4, NT = TXT * TYT;
        const int tid = threadIdx.x;
        const int tx = tid % TXT, ty = tid / TXT;
        TileEmit e;
        e.s = s;
        e.a = &a;
        e.cf = a.coef[sample];  // issued before the row loop, which hides its latency
        e.ox = tx * RX;
        e.oy = ty * RY;
        e.x0 = x0;
        e.y0 = y0;
        e.last = last;
        e.part = 0.0;
        e.ctx = tma_row_ctx<R>(a, sample, x0 + e.ox, y0 + e.oy, RY);
        TileAcc<RY, ALGO> t;
        tile_rows<R, RY, TXT, ALGO>(t, e, std::make_integer_sequence<int, RY + 2 * R>{});
        if (last) tma_tile_partial<NT>(a, sample, tile, e.part, red);
    }
}

// The update, projection and stores of a thread's RX x RY outputs from their disc sums acc,
// and the FP64 partial of the OoI when `last` (the weighted form).
template <int R, int RY, int TXT, int TYT>
__device__ __forceinline__ void tma_tile_epilogue(const float *s, const TmaArgs &a, int sample, int tile, int x0,
                                                  int y0, bool last, double *red, const StepCoef &cf,
                                                  const float (&acc)[RY][4]) {
    constexpr int RX = 4, R4 = (R + 3) & ~3, SW = 4 * TXT + 2 * R4, NT = TXT * TYT;
    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT, ox = tx * RX, oy = ty * RY;
    const TmaRowCtx ctx = tma_row_ctx<R>(a, sample, x0 + ox, y0 + oy, RY);
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < RY; ++j) {
        const float4 uc = *reinterpret_cast<const float4 *>(s + (oy + j + R) * SW + ox + R4);
        tma_emit_row<R>(a, ctx, cf, uc, make_float2(acc[j][0], acc[j][1]), make_float2(acc[j][2], acc[j][3]),
                        y0 + oy + j, x0 + ox, last, part);
    }
    if (last) tma_tile_partial<NT>(a, sample, tile, part, red);
}

// Weighted disc sums (ALGO 3), S_i = sum_z what(|z|) u_{i+z} for any radial kernel: per |dy|
// the R + 1 weights of |dx| = 0..R (zero beyond the disc's half-width) come from the table `wsm`
// in shared memory, and the dx loop runs in groups of four up to the row's half-width; each
// thread keeps its window of a staged row in registers and pairs the points +dx and -dx under
// one weight.  The dy loop is not unrolled (the code stays one row long for any R); dx, the
// output rows and columns are.
template <int R, int RY, int TXT, int TYT>
__device__ __forceinline__ void tma_tile_weighted(const float *s, const float *wsm, const TmaArgs &a, int sample,
                                                  int tile, int x0, int y0, bool last, double *red) {
    constexpr int RX = 4, R4 = (R + 3) & ~3, SW = 4 * TXT + 2 * R4, WIN = RX + 2 * R4;
    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT, ox = tx * RX, oy = ty * RY;
    const StepCoef cf = a.coef[sample];
    float acc[RY][RX];
#pragma unroll
    for (int j = 0; j < RY; ++j)
#pragma unroll
        for (int i = 0; i < RX; ++i) acc[j][i] = 0.f;
#pragma unroll 1
    for (int dy = -R; dy <= R; ++dy) {
        const int ady = dy < 0 ? -dy : dy;
        const float *wr = wsm + ady * (R + 1);
        float wv[R + 1];
#pragma unroll
        for (int q = 0; q <= R; ++q) wv[q] = wr[q];
        // half-width of the disc in this row: weights beyond it are zero, so the dx loop stops at
        // the first group of four that lies wholly outside (uniform across the CTA)
        int hw = (int)sqrtf((float)(R * R - ady * ady));
        while (hw * hw > R * R - ady * ady) --hw;
        while ((hw + 1) * (hw + 1) <= R * R - ady * ady) ++hw;
#pragma unroll
        for (int j = 0; j < RY; ++j) {
            const float4 *rowp = reinterpret_cast<const float4 *>(s + (oy + j + R + dy) * SW + ox);
            float v[WIN];
#pragma unroll
            for (int q = 0; q < WIN / 4; ++q) {
                const float4 t = rowp[q];
                v[4 * q + 0] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
#pragma unroll
            for (int i = 0; i < RX; ++i) acc[j][i] = fmaf(wv[0], v[R4 + i], acc[j][i]);
#pragma unroll
            for (int d0 = 1; d0 <= R; d0 += 4) {
                if (d0 > hw) break;
#pragma unroll
                for (int i = 0; i < RX; ++i) {
                    float t = acc[j][i];
#pragma unroll
                    for (int d = d0; d < d0 + 4 && d <= R; ++d) t = fmaf(wv[d], v[R4 + i + d] + v[R4 + i - d], t);
                    acc[j][i] = t;
                }
            }
        }
    }
    tma_tile_epilogue<R, RY, TXT, TYT>(s, a, sample, tile, x0, y0, last, red, cf, acc);
}

// STAGES = 2: the next item's copy is issued before computing the current one;
// STAGES = 1: it is issued after the current item is done (less shared memory per CTA,
// so more CTAs per SM overlap their copies with each other's compute).
template <int R, int RY, int TXT, int TYT, int ALGO, int STAGES>
__device__ __forceinline__ void tma_step_body(const CUtensorMap &src_map, const TmaArgs &a) {
    using C = TmaCfg<R, RY, TXT, TYT, STAGES>;
    constexpr int R4 = C::R4, NT = TXT * TYT;
    extern __shared__ unsigned char smem_raw[];
    float *base = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ double red[(NT + 31) / 32];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    float *wsm = base + STAGES * C::STAGE_FLOATS;  // ALGO 3: the weight table after the stages
    if constexpr (ALGO == 3)
        for (int i = tid; i < (R + 1) * (R + 1); i += NT) wsm[i] = a.wsq[i];
    __syncthreads();

    auto issue = [&](int item, int stage) {
        const int sample = item / a.tiles, tile = item - sample * a.tiles;
        const int x0 = (tile % a.tiles_x) * C::TX, y0 = (tile / a.tiles_x) * C::TY;
        mbar_expect_tx(&bars[stage], C::BOX_BYTES);
        // padded coordinates of the halo corner: (G + x0 - R4, G + y0 - R) = (x0, y0 + R4 - R)
        tma_load_3d(base + stage * C::STAGE_FLOATS, &src_map, &bars[stage], x0, y0 + R4 - R, sample);
    };

    int k = 0;
    int issued = 0;  // copies issued by thread 0 (item k's copy is copy number k)
    const int stride = gridDim.x;
    const int first = next_active(a, blockIdx.x, stride);
    if (tid == 0 && first < a.total) {
        issue(first, 0);
        issued = 1;
    }
    for (int item = first, nxt; item < a.total; item = nxt, ++k) {
        nxt = next_active(a, item + stride, stride);
        const int stage = STAGES == 2 ? (k & 1) : 0;
        const uint32_t parity = STAGES == 2 ? (uint32_t)((k >> 1) & 1) : (uint32_t)(k & 1);
        if (STAGES == 2 && tid == 0 && nxt < a.total) {
            issue(nxt, stage ^ 1);
            ++issued;
        }
        // bounded wait for this stage's copy
        long long spins = 0;
        while (!mbar_try_wait(&bars[stage], parity)) {
            if (++spins > kWaitLimit) {
                abort_flag = 1;
                break;
            }
        }
        __syncthreads();
        if (abort_flag) {
            // A copy did not land within the bound (only a copy that never completes can cause
            // it).  Report, then wait, again bounded, for every copy issued and not consumed
            // (items k .. issued - 1), so that none still targets this CTA's shared memory when
            // it exits unless that wait runs out as well.
            if (tid == 0) {
                atomicExch(a.status, 1);
                for (int j = k; j < issued; ++j) {
                    const int sj = STAGES == 2 ? (j & 1) : 0;
                    const uint32_t pj = STAGES == 2 ? (uint32_t)((j >> 1) & 1) : (uint32_t)(j & 1);
                    long long w = 0;
                    while (!mbar_try_wait(&bars[sj], pj) && ++w < kWaitLimit) {
                    }
                }
            }
            break;
        }
        const float *s = base + stage * C::STAGE_FLOATS;
        const int sample = item / a.tiles, tile = item - sample * a.tiles;
        const int x0 = (tile % a.tiles_x) * C::TX, y0 = (tile / a.tiles_x) * C::TY;
        const bool last = a.last || (a.steps_ps != nullptr && a.step == a.steps_ps[sample]);

        if constexpr (ALGO == 3)
            tma_tile_weighted<R, RY, TXT, TYT>(s, wsm, a, sample, tile, x0, y0, last, red);
        else
            tma_tile_compute<R, RY, TXT, TYT, ALGO>(s, a, sample, tile, x0, y0, last, red);
        __syncthreads();  // every thread is done with this stage before it is refilled
        if (STAGES == 1 && tid == 0 && nxt < a.total) {
            issue(nxt, 0);
            ++issued;
        }
    }
}

// The kernel, with the compiler's own register budget, and a variant whose register use
// is capped so that MINB CTAs fit on an SM.
template <int R, int RY, int TXT, int TYT, int ALGO, int STAGES = 2>
__global__ void __launch_bounds__(TXT *TYT) step_tma_kernel(const __grid_constant__ CUtensorMap src_map,
                                                            TmaArgs a) {
    tma_step_body<R, RY, TXT, TYT, ALGO, STAGES>(src_map, a);
}

template <int R, int RY, int TXT, int TYT, int ALGO, int STAGES, int MINB>
__global__ void __launch_bounds__(TXT *TYT, MINB) step_tma_kernel_capped(const __grid_constant__ CUtensorMap src_map,
                                                                         TmaArgs a) {
    tma_step_body<R, RY, TXT, TYT, ALGO, STAGES>(src_map, a);
}

template <int R, int RY, int TXT, int TYT, int ALGO, int STAGES, int MINB>
constexpr auto tma_kernel_ptr() {
    if constexpr (MINB <= 1)
        return &step_tma_kernel<R, RY, TXT, TYT, ALGO, STAGES>;
    else
        return &step_tma_kernel_capped<R, RY, TXT, TYT, ALGO, STAGES, MINB>;
}

// Copy unpadded fields [ns][n][n] into padded scratch [ns][P][P] including the frame: the
// periodic images, or the collar value uI when `collar` (defined in nlch_solver.cu).
__global__ void pad_fields_kernel(const float *u, float *dst, int n, int G, size_t ns, int collar, float uI);

// --------------------------------------------------------------------------- host side
// Tile shapes (rows per thread RY, threads along x TXT, threads along y TYT):
//   variant 0: 4 x 16 outputs per thread, 64 x 128 tile, 128 threads
//   variant 1: 4 x 8 outputs per thread,  64 x 128 tile, 256 threads
//   variant 2: 4 x 8 outputs per thread,  64 x 64 tile,  128 threads
//   variants 3, 4: shapes 0 and 1 with a single shared-memory stage
//   variant 5: variant 4 with at most 64 registers per thread (4 CTAs per SM)
//   variant 6: 4 x 16 outputs per thread, 128 x 128 tile, 256 threads, one stage, <= 128 registers
//   variant 7: 4 x 16 outputs per thread, 64 x 128 tile, 128 threads, one stage, <= 168 registers
//   variant 8: 4 x 16 outputs per thread, 64 x 64 tile, 64 threads, one stage
//   variant 9: variant 8 with at most 128 registers per thread (8 CTAs per SM)
//   variant 10: 4 x 16 outputs per thread, 128 x 64 tile, 128 threads, one stage
constexpr int kTmaVariants = 11;
// The weighted form (ALGO 3) runs one more shape: 4 x 4 outputs per thread, 64 x 64 tile,
// 256 threads, one stage (its window and weight registers leave room for only 4 output rows).
constexpr int kTmaWeighted = kTmaVariants;

template <int V>
struct TmaShape;
template <>
struct TmaShape<0> {
    static constexpr int RY = 16, TXT = 16, TYT = 8, STAGES = 2, MINB = 1;
};
template <>
struct TmaShape<1> {
    static constexpr int RY = 8, TXT = 16, TYT = 16, STAGES = 2, MINB = 1;
};
template <>
struct TmaShape<2> {
    static constexpr int RY = 8, TXT = 16, TYT = 8, STAGES = 2, MINB = 1;
};
template <>
struct TmaShape<3> {
    static constexpr int RY = 16, TXT = 16, TYT = 8, STAGES = 1, MINB = 1;
};
template <>
struct TmaShape<4> {
    static constexpr int RY = 8, TXT = 16, TYT = 16, STAGES = 1, MINB = 1;
};
template <>
struct TmaShape<5> {
    static constexpr int RY = 8, TXT = 16, TYT = 16, STAGES = 1, MINB = 4;
};
template <>
struct TmaShape<6> {
    static constexpr int RY = 16, TXT = 32, TYT = 8, STAGES = 1, MINB = 2;
};
template <>
struct TmaShape<7> {
    static constexpr int RY = 16, TXT = 16, TYT = 8, STAGES = 1, MINB = 3;
};
template <>
struct TmaShape<8> {
    static constexpr int RY = 16, TXT = 16, TYT = 4, STAGES = 1, MINB = 1;
};
template <>
struct TmaShape<9> {
    static constexpr int RY = 16, TXT = 16, TYT = 4, STAGES = 1, MINB = 8;
};
template <>
struct TmaShape<10> {
    static constexpr int RY = 16, TXT = 32, TYT = 4, STAGES = 1, MINB = 1;
};
template <>
struct TmaShape<kTmaWeighted> {
    static constexpr int RY = 4, TXT = 16, TYT = 16, STAGES = 1, MINB = 1;
};

typedef mfmc_status (*TmaFn)(const CUtensorMap &, const TmaArgs &, int grid, cudaStream_t);

struct TmaVariant {
    int tx, ty, sw, sh, threads;
    size_t smem;
    TmaFn fn[4];  // [algo]: unused, prefix, prefix-Kahan, weighted
    int (*blocks_per_sm)();
};

struct TmaLauncher {
    TmaVariant v[kTmaVariants + 1];  // [kTmaWeighted]: the weighted form (fn[3])
};

template <int R, int V, int ALGO>
mfmc_status launch_tma(const CUtensorMap &map, const TmaArgs &a, int grid, cudaStream_t st) {
    using T = TmaShape<V>;
    using C = TmaCfg<R, T::RY, T::TXT, T::TYT, T::STAGES>;
    auto kern = tma_kernel_ptr<R, T::RY, T::TXT, T::TYT, ALGO, T::STAGES, T::MINB>();
    constexpr size_t smem = C::SMEM + (ALGO == 3 ? (size_t)(R + 1) * (R + 1) * sizeof(float) : 0);
    // set before every launch: the attribute is per device, and the call is cheap
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, T::TXT * T::TYT, smem, st>>>(map, a);
    MFMC_LAUNCHED("tma_step launch 1");
    return MFMC_OK;
}

template <int R, int V>
int tma_blocks_per_sm() {
    using T = TmaShape<V>;
    using C = TmaCfg<R, T::RY, T::TXT, T::TYT, T::STAGES>;
    constexpr int ALGO = V == kTmaWeighted ? 3 : 1;
    constexpr size_t smem = C::SMEM + (ALGO == 3 ? (size_t)(R + 1) * (R + 1) * sizeof(float) : 0);
    if constexpr (V != kTmaWeighted && T::RY > 16 && R > 16) {
        return 1;  // not built (see make_tma_variant)
    } else {
        auto k = tma_kernel_ptr<R, T::RY, T::TXT, T::TYT, ALGO, T::STAGES, T::MINB>();
        int per = 0;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, T::TXT * T::TYT, smem);
        (void)cudaGetLastError();  // a failed query must not be reported by a later launch check
        return e == cudaSuccess && per > 0 ? per : 1;
    }
}

template <int R, int V, bool KAHAN>
TmaVariant make_tma_variant() {
    using T = TmaShape<V>;
    using C = TmaCfg<R, T::RY, T::TXT, T::TYT, T::STAGES>;
    TmaVariant L;
    L.tx = C::TX;
    L.ty = C::TY;
    L.sw = C::SW;
    L.sh = C::SH;
    L.threads = T::TXT * T::TYT;
    L.smem = C::SMEM;
    L.fn[0] = nullptr;
    if constexpr (V == kTmaWeighted) {
        L.fn[1] = L.fn[2] = nullptr;
        L.fn[3] = &launch_tma<R, V, 3>;
    } else if constexpr (T::RY > 16 && R > 16) {
        // 32-row blocks are built for horizons up to 16 only (the unrolled row loop of a
        // wider horizon is too long)
        L.fn[1] = L.fn[2] = L.fn[3] = nullptr;
    } else {
        L.fn[1] = &launch_tma<R, V, 1>;
        L.fn[3] = nullptr;
        if constexpr (KAHAN) {
            L.fn[2] = &launch_tma<R, V, 2>;
        } else {
            L.fn[2] = nullptr;
        }
    }
    L.blocks_per_sm = &tma_blocks_per_sm<R, V>;
    return L;
}

template <int R>
TmaLauncher make_tma_launcher() {
    TmaLauncher L;
    L.v[0] = make_tma_variant<R, 0, true>();
    L.v[1] = make_tma_variant<R, 1, false>();
    L.v[2] = make_tma_variant<R, 2, false>();
    L.v[3] = make_tma_variant<R, 3, false>();
    L.v[4] = make_tma_variant<R, 4, false>();
    L.v[5] = make_tma_variant<R, 5, false>();
    L.v[6] = make_tma_variant<R, 6, false>();
    L.v[7] = make_tma_variant<R, 7, false>();
    L.v[8] = make_tma_variant<R, 8, false>();
    L.v[9] = make_tma_variant<R, 9, false>();
    L.v[10] = make_tma_variant<R, 10, false>();
    L.v[kTmaWeighted] = make_tma_variant<R, kTmaWeighted, false>();
    return L;
}

// Defined in the per-R translation units.
const TmaLauncher *tma_launcher(int R);

}  // namespace mfmc
