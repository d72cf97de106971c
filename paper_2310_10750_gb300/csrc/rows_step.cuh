// Row-streaming step kernel (constant kernel, R <= 8, n % 128 == 0, n <= 2048).
//
// A CTA of 16 warps (fewer when 16 is no multiple of n / 128) streams whole rows of GS
// consecutive samples down a range of rows: warp w takes the 128-column strip w % (n / 128) of
// sample w / (n / 128) of its group, lane l the strip's columns 4l .. 4l+3.  The batch's rows,
// ordered by (sample group, row), are split evenly over the CTAs (or into fixed bands taken in
// turn); a CTA's range is cut into segments at group boundaries, and each segment's rows are
// walked downwards together with an R-row halo above and below (always downwards: each output's
// disc rows are then summed top to bottom whatever the split, so results do not depend on it).
// The rows arrive through a ring of shared-memory
// chunks: one TMA box per chunk carries CH whole ghost-framed rows (P = n + 2 R4 floats, read
// through a four-dimensional view that splits a row into k pieces of at most 256 floats) of
// all GS samples, so every byte of a field is fetched once; the copy of the next chunk is
// issued when a chunk is entered.  All warps run the same instructions on the same rows.
//
// From each staged row a lane forms its window's centre sums and one segment sum per distinct
// disc-row half-width, and adds each to the 2R + 1 output rows that the row touches; the
// accumulators (packed FP32 pairs) form a ring of 2R + 1 slots, so every staged row is summed
// once per segment.  After staged row q the output row q - 2R is complete and is finished at
// once (update, projection, store with ghost images).  The row loop is unrolled by the ring
// period 2R + 1, which keeps every slot index static.  The OoI is reduced afterwards from the
// final fields (rows_ooi_kernel), so it does not depend on how the rows were split.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "tma_step.cuh"

namespace mfmc {

struct RowsArgs {
    TmaArgs t;             // outputs, coefficients, status, step counts, step, n, P, periodic
    int ns;                // samples
    int gs;                // samples per CTA
    int strips;            // n / 128: warps per sample
    long long rows;        // groups * n: the batch's rows in (group, row) order
    int band;              // rows per work range; 0: rows / groups, one range per group
    int stage_floats;      // gs * CH * P
    int ng;                // independent warp groups per CTA (each gs samples)
};

template <int R>
struct RowsCfg {
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int CH = 8;                         // rows per chunk
    // a stage is refilled (with the chunk after the next) once no row of it is read again: the
    // oldest row still read is the centre row R rows back, so 2 + ceil(R / CH) stages suffice
    static constexpr int NSTG = 2 + (R + CH - 1) / CH;
    // accumulator ring slots: the 2R + 1 output rows a staged row touches (larger rings that
    // are multiples of CH would make chunk boundaries static but spill registers)
    static constexpr int S = 2 * R + 1;
    static constexpr int MAXW = 16;                      // warps per CTA at most
    static constexpr int MAXG = 4;                       // warp groups per CTA at most
};

// Barriers of one warp group (named barrier id, nthreads threads; id 0 is the CTA's).
__device__ __forceinline__ bool group_sync_and(int id, int nthreads, bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// A segment of the walk: sample group, first row and rows (len = 0: end of the walk).
struct RowsSegInfo {
    int group, y0, len;
};

// The CTA's walk over its row ranges (thread 0 only; results go through shared memory).
struct RowsSegIter {
    long long q, qend;     // the part of the current range still to walk
    long long range;       // index of the current range
    long long nct;
    __device__ void set_range(const RowsArgs &a) {
        if (a.band > 0) {
            q = range * a.band;
            qend = q + a.band < a.rows ? q + a.band : a.rows;
        } else {
            const long long base = a.rows / nct, rem = a.rows % nct;
            q = base * range + (range < rem ? range : rem);
            qend = q + base + (range < rem ? 1 : 0);
        }
        if (q > a.rows) q = qend = a.rows;
    }
    __device__ void init(const RowsArgs &a, long long id, long long count) {
        nct = count;
        range = id;
        set_range(a);
    }
    // The next segment with an active sample, in walk order; len = 0 at the end.
    __device__ RowsSegInfo next(const RowsArgs &a) {
        const int n = a.t.n;
        RowsSegInfo s;
        for (;;) {
            if (q >= qend) {
                range += nct;
                if (a.band == 0 || range * a.band >= a.rows) {
                    s.group = s.y0 = s.len = 0;
                    return s;
                }
                set_range(a);
                continue;
            }
            const long long col = q / n;
            const long long hi = (col + 1) * n < qend ? (col + 1) * n : qend;
            s.group = (int)col;
            s.y0 = (int)(q - col * n);
            s.len = (int)(hi - q);
            q = hi;
            bool any = false;
            for (int w = 0; w < a.gs; ++w) {
                const int smp = a.gs * s.group + w;
                any = any || (smp < a.ns && (a.t.steps_ps == nullptr || a.t.step <= a.t.steps_ps[smp]));
            }
            if (any) return s;
        }
    }
};

// Shared state of a CTA: the walk, the producer's position and two segment slots (the
// consumer's current segment and the next one).
struct RowsShared {
    RowsSegIter it;
    RowsSegInfo seg[2];
    int pslot, pc, pnch;   // producer: segment slot, next chunk in it, its chunk count
    int pg;                // chunks issued
};

template <int R>
__device__ __noinline__ void rows_issue(const RowsArgs &a, RowsShared &sh, const CUtensorMap *map, float *ring,
                                        uint64_t *bar) {
    using C = RowsCfg<R>;
    if (sh.pc >= sh.pnch) {
        sh.pslot ^= 1;
        sh.pnch = sh.seg[sh.pslot].len > 0 ? (sh.seg[sh.pslot].len + 2 * R + C::CH - 1) / C::CH : 0;
        sh.pc = 0;
        if (sh.pnch == 0) return;
    }
    const RowsSegInfo &s = sh.seg[sh.pslot];
    const int st = sh.pg % C::NSTG;
    // lattice rows of chunk c: y0 - R + c CH + [0, CH); padded row = G + lattice row (G = R4)
    const int ylo = s.y0 - R + sh.pc * C::CH;
    mbar_expect_tx(&bar[st], (uint32_t)a.stage_floats * sizeof(float));
    tma_load_4d(ring + (size_t)st * a.stage_floats, map, &bar[st], 0, 0, C::R4 + ylo, a.gs * s.group);
    ++sh.pc;
    ++sh.pg;
}

// Per-segment state of a warp.
struct RowsSeg {
    const float *win0;   // the lane's window start in its sample's first row of stage 0
    int bid, bthreads;   // the warp group's named barrier and its threads
    bool leader;         // the group's first thread: issues the copies and walks the segments
    int g0;              // stream index of the segment's first chunk
    int nrows;           // rows walked: len + 2R
    int sample;
    // outputs: the next output row's four values go to out (advanced by ostride per row), its
    // ghost column image to out + gdelta, and for lattice rows yr < G or yr >= n - G also to
    // the ghost row image (out +- n P); flags say which of these exist
    float *out;
    long long gdelta;
    int ostride, yr;
    unsigned flags;
    float2 nc0, c1, c2;  // step coefficients (-c0, c1, c2) in both halves of a pair
};

enum : unsigned { kRowsActive = 1u, kRowsGhostCol = 2u, kRowsGhostRows = 4u };

// The update and projection of one output row of a lane (four columns) from its disc sums
// (s01, s23) and centre values uc, and its stores (Eq. nonl_CH_nm with beta2 = 0 and the
// projection of Eq. potential_obstacle): sd = fma(-c0, u, S), v = u + fma(c1, sd, c2 u),
// u_new = min(1, max(-1, v)), each packed FP32 pair rounding exactly like the scalar operations.
template <int R>
__device__ __forceinline__ void rows_emit(RowsSeg &sg, unsigned fl, float4 uc, float2 s01, float2 s23, int n, int P) {
    constexpr int G = (R + 3) & ~3;
    const float2 u01 = make_float2(uc.x, uc.y), u23 = make_float2(uc.z, uc.w);
    const float2 v01 = __fadd2_rn(u01, __ffma2_rn(sg.c1, __ffma2_rn(sg.nc0, u01, s01), __fmul2_rn(sg.c2, u01)));
    const float2 v23 = __fadd2_rn(u23, __ffma2_rn(sg.c1, __ffma2_rn(sg.nc0, u23, s23), __fmul2_rn(sg.c2, u23)));
    const float4 val = make_float4(fminf(1.f, fmaxf(-1.f, v01.x)), fminf(1.f, fmaxf(-1.f, v01.y)),
                                   fminf(1.f, fmaxf(-1.f, v23.x)), fminf(1.f, fmaxf(-1.f, v23.y)));
    *reinterpret_cast<float4 *>(sg.out) = val;
    if (fl & kRowsGhostCol) *reinterpret_cast<float4 *>(sg.out + sg.gdelta) = val;
    if ((fl & kRowsGhostRows) && (unsigned)(sg.yr - G) >= (unsigned)(n - 2 * G)) {
        const long long off = (long long)(sg.yr < G ? n : -n) * P;  // the row's periodic image
        *reinterpret_cast<float4 *>(sg.out + off) = val;
        if (fl & kRowsGhostCol) *reinterpret_cast<float4 *>(sg.out + off + sg.gdelta) = val;
    }
}

template <int R>
struct RowsAcc {
    float2 acc[RowsCfg<R>::S][2];  // slot j mod S: output row j (at most 2R + 1 live at a time)
    const float *rp, *cp;          // the lane's window in the staged row, its centre R rows back
    int cst;                       // stage of the centre row's chunk
};

__device__ __forceinline__ constexpr int rows_mod(int a, int m) { return ((a % m) + m) % m; }

template <int R>
struct RowsPlan {
    static constexpr DiscClasses<R> cls{};
    __host__ __device__ static constexpr bool serves(int dy, int c) { return cls.of[dy < 0 ? -dy : dy] == c; }
};

// Adds the class-c segment sums of staged row (ring position K) to every ring slot that the
// class serves: dy with cls.of[|dy|] == c, output row q - R - dy in slot (K - R - dy) mod S.
// The output row's first staged row (dy = -R) starts its slot.
template <int R, int K, int c, int... D>
__device__ __forceinline__ void rows_class(RowsAcc<R> &t, const RowWin<R> &win, std::integer_sequence<int, D...>) {
    float h[4];
    class_sums<R, RowsPlan<R>::cls.width[c]>(win, h);
    const float2 h01 = make_float2(h[0], h[1]), h23 = make_float2(h[2], h[3]);
    auto add = [&](auto dc) {
        constexpr int dy = decltype(dc)::value - R;
        if constexpr (RowsPlan<R>::serves(dy, c)) {
            constexpr int slot = rows_mod(K - R - dy, RowsCfg<R>::S);
            if constexpr (dy == -R) {
                t.acc[slot][0] = h01;
                t.acc[slot][1] = h23;
            } else {
                t.acc[slot][0] = __fadd2_rn(t.acc[slot][0], h01);
                t.acc[slot][1] = __fadd2_rn(t.acc[slot][1], h23);
            }
        }
    };
    (add(std::integral_constant<int, D>{}), ...);
}

template <int R, int K, int... Cs>
__device__ __forceinline__ void rows_classes(RowsAcc<R> &t, const RowWin<R> &win, std::integer_sequence<int, Cs...>) {
    (rows_class<R, K, Cs>(t, win, std::make_integer_sequence<int, 2 * R + 1>{}), ...);
}

// Staged row q = q0 + K of the segment (q0 a multiple of S, K static: the ring position).
// Returns false when a chunk wait ran out of its bound.
template <int R, int K>
__device__ __forceinline__ bool rows_row(RowsAcc<R> &t, const RowsArgs &a, RowsSeg &sg, int q0, RowsShared &sh,
                                         const CUtensorMap *map, float *ring, uint64_t *bar) {
    using C = RowsCfg<R>;
    const int q = q0 + K;
    t.rp += a.t.P;
    t.cp += a.t.P;
    if (q % C::CH == 0) {
        const int g = sg.g0 + q / C::CH;
        const int st = g % C::NSTG;
        t.rp = sg.win0 + st * a.stage_floats;
        long long spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&bar[st], (uint32_t)((g / C::NSTG) & 1)))
            if (++spins > kWaitLimit) {
                ok = false;
                break;
            }
        // every thread of the group is past the rows of the stage that the next copy overwrites
        if (!group_sync_and(sg.bid, sg.bthreads, ok)) return false;
        if (sg.leader) rows_issue<R>(a, sh, map, ring, bar);
    }
    // the centre row q - R enters a new chunk: the stage after the previous centre chunk's
    if ((R % C::CH == 0 ? q % C::CH == 0 : (q - R) % C::CH == 0) && q >= R) {
        t.cst = t.cst + 1 == C::NSTG ? 0 : t.cst + 1;
        t.cp = sg.win0 + t.cst * a.stage_floats + C::R4;
    }
    RowWin<R> win;
    row_window<R>(t.rp, win);
    rows_classes<R, K>(t, win, std::make_integer_sequence<int, RowsPlan<R>::cls.count>{});
    if (q >= 2 * R) {  // output row q - 2R is complete
        const unsigned fl = opaque_u32(sg.flags);
        if (fl & kRowsActive) {
            constexpr int slot = rows_mod(K - 2 * R, C::S);
            const float4 uc = *reinterpret_cast<const float4 *>(t.cp);  // its centre row, q - R
            rows_emit<R>(sg, fl, uc, t.acc[slot][0], t.acc[slot][1], a.t.n, a.t.P);
        }
        sg.out += sg.ostride;
        ++sg.yr;
    }
    return true;
}

template <int R, int... Ks>
__device__ __forceinline__ bool rows_block(RowsAcc<R> &t, const RowsArgs &a, RowsSeg &sg, int q0,
                                           RowsShared &sh, const CUtensorMap *map, float *ring, uint64_t *bar,
                                           int *gfail, std::integer_sequence<int, Ks...>) {
    using C = RowsCfg<R>;
    bool ok = true;
    auto one = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (ok && q0 + K < sg.nrows) {
            ok = rows_row<R, K>(t, a, sg, q0, sh, map, ring, bar);
            if (!ok) *gfail = sg.g0 + (q0 + K) / C::CH;
        }
    };
    (one(std::integral_constant<int, Ks>{}), ...);
    return ok;
}

template <int R>
__global__ void __launch_bounds__(RowsCfg<R>::MAXW * 32, 1) step_rows_kernel(const __grid_constant__ CUtensorMap map,
                                                                           RowsArgs a) {
    using C = RowsCfg<R>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[C::MAXG][C::NSTG];
    __shared__ RowsShared shs[C::MAXG];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp groups: a.gs samples x a.strips strips each, independent rings and barriers
    const int gw = a.gs * a.strips, gid = warp / gw, wig = warp - gid * gw;
    const int sl = wig / a.strips, strip = wig - sl * a.strips;  // sample in the group, strip
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127)) +
                  (size_t)gid * C::NSTG * a.stage_floats;
    uint64_t *bar = bars[gid];
    RowsShared &sh = shs[gid];
    const bool leader = (threadIdx.x - 32 * gw * gid) == 0;
    if (leader) {
        for (int i = 0; i < C::NSTG; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.it.init(a, (long long)blockIdx.x * a.ng + gid, (long long)gridDim.x * a.ng);
        sh.seg[0] = sh.it.next(a);
        sh.seg[1] = sh.it.next(a);
        sh.pslot = 1;  // the first issue advances to slot 0
        sh.pc = sh.pnch = 0;
        sh.pg = 0;
        rows_issue<R>(a, sh, &map, ring, bar);
    }
    __syncthreads();
    RowsAcc<R> t;
#pragma unroll
    for (int k = 0; k < C::S; ++k) t.acc[k][0] = t.acc[k][1] = make_float2(0.f, 0.f);

    RowsSeg sg;
    sg.win0 = ring + sl * C::CH * a.t.P + 128 * strip + 4 * lane;
    sg.bid = 1 + gid;
    sg.bthreads = 32 * gw;
    sg.leader = leader;
    sg.g0 = 0;
    int gfail = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
        const RowsSegInfo s = sh.seg[k & 1];
        if (s.len == 0) break;
        sg.nrows = s.len + 2 * R;
        // the centre row q - R enters chunk 0 at q = R (rows q < R have no centre in use): start
        // one stage before the segment's first chunk
        t.cst = (sg.g0 + C::NSTG - 1) % C::NSTG;
        t.rp = t.cp = sg.win0;
        sg.sample = a.gs * s.group + sl;
        {
            const int n = a.t.n, P = a.t.P, x = 128 * strip + 4 * lane;
            const bool active =
                sg.sample < a.ns && (a.t.steps_ps == nullptr || a.t.step <= a.t.steps_ps[sg.sample]);
            const int smp = active ? sg.sample : 0;
            const StepCoef cf = a.t.coef[smp];
            sg.nc0 = make_float2(-cf.c0, -cf.c0);
            sg.c1 = make_float2(cf.c1, cf.c1);
            sg.c2 = make_float2(cf.c2, cf.c2);
            sg.yr = s.y0;
            sg.flags = active ? kRowsActive : 0u;
            sg.gdelta = 0;
            if (a.t.dst_plain) {  // the caller's unpadded field (last step): no ghost images
                sg.out = a.t.dst_plain + (size_t)smp * n * n + (size_t)s.y0 * n + x;
                sg.ostride = n;
            } else {
                sg.out = a.t.dst + (size_t)smp * P * P + (size_t)(C::R4 + s.y0) * P + C::R4 + x;
                sg.ostride = P;
                if (a.t.periodic) {
                    // the lane's columns have a periodic image in the frame, n columns to the right
                    // when x < G and n columns to the left when x >= n - G
                    if (x < C::R4 || x >= n - C::R4) {
                        sg.flags |= kRowsGhostCol;
                        sg.gdelta = x < C::R4 ? n : -n;
                    }
                    sg.flags |= kRowsGhostRows;
                }
            }
        }
        for (int q0 = 0; ok && q0 < sg.nrows; q0 += C::S)
            ok = rows_block<R>(t, a, sg, q0, sh, &map, ring, bar, &gfail, std::make_integer_sequence<int, C::S>{});
        sg.g0 += (sg.nrows + C::CH - 1) / C::CH;
        group_sync(sg.bid, sg.bthreads);  // every thread of the group has read slot k & 1
        if (ok && leader) sh.seg[k & 1] = sh.it.next(a);
        group_sync(sg.bid, sg.bthreads);
    }
    if (!ok && leader) {
        // A chunk wait ran out of its bound (only a copy that never lands can cause it): report,
        // then wait, again bounded, for each copy issued and not consumed, so that none still
        // targets the ring when the CTA exits unless that wait runs out as well.
        atomicExch(a.t.status, 1);
        for (int g = gfail; g < sh.pg; ++g) {
            long long spins = 0;
            while (!mbar_try_wait(&bar[g % C::NSTG], (uint32_t)((g / C::NSTG) & 1)) && ++spins < kWaitLimit) {
            }
        }
    }
}

// FP64 sum of every (sample, strip, row) of the final fields into partials[ns][strips][n] (lane
// sums of four values, then a fixed shuffle tree), read from the unpadded fields `plain` when
// given, else from the ghost-framed buffer that holds each sample's last step: A after an odd
// number of steps, B after an even one (steps_ps: per-sample step counts, or nsteps for all).
__global__ void rows_ooi_kernel(const float *plain, const float *padA, const float *padB, const int *steps_ps,
                                int nsteps, int n, int P, int G, int strips, size_t ns, double *partials);

// Geometry of the row-streaming kernel for a lattice: samples per CTA, warps, the split of a
// padded row into k pieces for the tensor map, and the dynamic shared memory.
struct RowsGeom {
    int strips, gs, warps, k, P, stage_floats;
    size_t smem;
};

struct RowsLauncher {
    int ch, nstg;
    mfmc_status (*fn)(const CUtensorMap &, const RowsArgs &, int grid, int threads, size_t smem, cudaStream_t);
    int (*blocks_per_sm)(int threads, size_t smem);
};

template <int R>
mfmc_status launch_rows(const CUtensorMap &map, const RowsArgs &a, int grid, int threads, size_t smem,
                        cudaStream_t st) {
    auto kern = step_rows_kernel<R>;
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, st>>>(map, a);
    MFMC_LAUNCHED("rows_step launch");
    return MFMC_OK;
}

template <int R>
int rows_blocks_per_sm(int threads, size_t smem) {
    auto kern = step_rows_kernel<R>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    (void)cudaGetLastError();  // a failed query must not be reported by a later launch check
    return e == cudaSuccess && per > 0 ? per : 1;
}

template <int R>
RowsLauncher make_rows_launcher() {
    RowsLauncher L;
    L.ch = RowsCfg<R>::CH;
    L.nstg = RowsCfg<R>::NSTG;
    L.fn = &launch_rows<R>;
    L.blocks_per_sm = &rows_blocks_per_sm<R>;
    return L;
}

// Defined in the per-R translation units (R <= 8).
const RowsLauncher *rows_launcher(int R);

}  // namespace mfmc
