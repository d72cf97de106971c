// Row-streaming step kernel (constant kernel, periodic lattice, R <= 8, n % 128 == 0, n <= 2048).
//
// A CTA of 16 warps (fewer when 16 is no multiple of n / 128) streams whole rows of GS
// consecutive samples down a range of rows: warp w takes the 128-column strip w % (n / 128) of
// sample w / (n / 128) of its group, lane l the strip's columns 4l .. 4l+3.  The batch's rows,
// ordered by (sample group, row), are split over the CTAs so that every CTA walks about as many
// rows, its halo rows included (or into fixed bands taken in turn); a CTA's range is cut into
// segments at group boundaries, and each segment's rows are walked downwards together with an
// R-row halo above and below (always downwards: each output's disc rows are then summed top to
// bottom whatever the split, so results do not depend on it).
//
// The fields are plain [sample][n][n] arrays: no ghost frame.  The rows arrive through a ring
// of shared-memory chunks, one TMA box per chunk carrying CH whole rows of all GS samples
// (stored [row][sample][n]; a four-dimensional view splits a row into k pieces of at most 256
// floats), so every byte of a field is fetched once.  The periodic images are taken on the fly:
// a chunk's lattice rows wrap modulo n in the copy's row coordinate (a chunk that straddles row
// 0 or row n is fetched row by row through a second view), and the lanes whose window crosses
// column 0 or column n read those float4s n columns away in the same staged row.  The copy of
// the next chunk is issued when a chunk is entered.  All warps run the same instructions on
// the same rows.
//
// From each staged row a lane forms its window's centre sums and one segment sum per distinct
// disc-row half-width, and adds each to the 2R + 1 output rows that the row touches; the
// accumulators (packed FP32 pairs) form a ring of 2R + 1 slots, so every staged row is summed
// once per segment.  After staged row q the output row q - 2R is complete and is finished at
// once (update, projection, store).  The row loop is unrolled by the ring period 2R + 1, which
// keeps every slot index static.  The OoI is reduced afterwards from the final fields
// (rows_ooi_kernel), so it does not depend on how the rows were split.
//
// Consecutive steps are launched as programmatic dependents: a step's CTAs set up their
// barriers and walk while the previous step drains, and wait for its completion
// (griddepcontrol.wait) before the first copy.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "tma_step.cuh"

namespace mfmc {

struct RowsArgs {
    TmaArgs t;             // destination (t.dst, plain fields), coefficients, status, step counts, step, n
    int ns;                // samples
    int gs;                // samples per CTA
    int strips;            // n / 128: warps per sample
    long long rows;        // groups * n: the batch's rows in (group, row) order
    int band;              // rows per work range; 0: an even split of rows and halos over the CTAs
    int halo;              // 2R: the rows a segment reads beyond its outputs
    int stage_floats;      // CH * gs * n
    int pitch;             // gs * n: floats from one staged row of a sample to its next
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

// The CTA's walk over its row ranges (one thread at a time; results go through shared memory).
// 32-bit arithmetic: the host keeps every walk-cost position below 2^31.
struct RowsSegIter {
    int q, qend;     // the part of the current range still to walk
    int range;       // index of the current range
    int nct;
    // Without bands the split is even in a walk-cost space where each group counts n + 2R
    // rows: its 2R halo rows of the group's first segment, then its n rows.  A range that
    // starts a new segment inside the group (at a cut or a group boundary) therefore walks 2R
    // rows more than it outputs and every range walks at most its share + 2R rows.
    __device__ static int walk_to_row(const RowsArgs &a, int v) {
        const int V = a.t.n + a.halo, g = v / V, o = v - g * V - a.halo;
        return g * a.t.n + (o > 0 ? o : 0);
    }
    __device__ void set_range(const RowsArgs &a) {
        const int rows = (int)a.rows;
        if (a.band > 0) {
            q = range * a.band;
            qend = q + a.band < rows ? q + a.band : rows;
        } else {
            const int total = rows / a.t.n * (a.t.n + a.halo);
            const int base = total / nct, rem = total % nct;
            const int vb = base * range + (range < rem ? range : rem);
            q = walk_to_row(a, vb);
            qend = walk_to_row(a, vb + base + (range < rem ? 1 : 0));
        }
        if (q > rows) q = qend = rows;
    }
    __device__ void init(const RowsArgs &a, int id, int count) {
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
                if (a.band == 0 || (long long)range * a.band >= a.rows) {
                    s.group = s.y0 = s.len = 0;
                    return s;
                }
                set_range(a);
                continue;
            }
            const int col = q / n;
            const int hi = (col + 1) * n < qend ? (col + 1) * n : qend;
            s.group = col;
            s.y0 = q - col * n;
            s.len = hi - q;
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

// Shared state of a CTA: the walk, the producer's position and three segment slots (segment k
// in slot k mod 3: the consumers' current one and the next two).
struct RowsShared {
    RowsSegIter it;
    RowsSegInfo seg[3];
    int pslot, pc, pnch;   // producer: segment slot, next chunk in it, its chunk count
    int pg;                // chunks issued
};

// Issues the copy of the next chunk of the walk (thread 0).  map: boxes of CH rows; map1: boxes
// of one row, for the chunks that straddle row 0 or row n.
template <int R>
__device__ __noinline__ void rows_issue(const RowsArgs &a, RowsShared &sh, const CUtensorMap *map,
                                        const CUtensorMap *map1, float *ring, uint64_t *bar) {
    using C = RowsCfg<R>;
    if (sh.pc >= sh.pnch) {
        sh.pslot = sh.pslot == 2 ? 0 : sh.pslot + 1;
        sh.pnch = sh.seg[sh.pslot].len > 0 ? (sh.seg[sh.pslot].len + 2 * R + C::CH - 1) / C::CH : 0;
        sh.pc = 0;
        if (sh.pnch == 0) return;
    }
    const RowsSegInfo &s = sh.seg[sh.pslot];
    const int st = sh.pg % C::NSTG, n = a.t.n;
    // lattice rows of chunk c: y0 - R + c CH + [0, CH), taken modulo n (-R <= y < n + R + CH)
    const int ylo = s.y0 - R + sh.pc * C::CH;
    float *dst = ring + (size_t)st * a.stage_floats;
    mbar_expect_tx(&bar[st], (uint32_t)a.stage_floats * sizeof(float));
    if ((ylo < 0 && ylo + C::CH > 0) || (ylo < n && ylo + C::CH > n)) {
        for (int r = 0; r < C::CH; ++r) {  // the chunk straddles a periodic seam: row by row
            const int y = ylo + r;
            tma_load_4d(dst + (size_t)r * a.pitch, map1, &bar[st], 0, 0, a.gs * s.group, y < 0 ? y + n : (y >= n ? y - n : y));
        }
    } else {
        tma_load_4d(dst, map, &bar[st], 0, 0, a.gs * s.group, ylo < 0 ? ylo + n : (ylo >= n ? ylo - n : ylo));
    }
    ++sh.pc;
    ++sh.pg;
}

// Per-segment state of a warp.
template <int R>
struct RowsSeg {
    static constexpr int NQ = RowWin<R>::WIN / 4, QC = RowWin<R>::R4 / 4;
    const float *win0;   // the lane's window start (column x - R4, unwrapped) in its sample's first row of stage 0
    int wd[NQ];          // per float4 of the window: 0, or +-n where it crosses column 0 or n (never at QC)
    int bid, bthreads;   // the warp group's named barrier and its threads
    bool leader;         // the group's first thread: walks the segments
    int tig, gw;         // the thread's index in its group, the group's warps
    int kseg;            // index of the current segment (its slot: kseg mod 3)
    int g0;              // stream index of the segment's first chunk
    int nrows;           // rows walked: len + 2R
    float *out;          // the next output row's four values (rows advance by n)
    unsigned flags;
    float2 nc0, c1, c2;  // step coefficients (-c0, c1, c2) in both halves of a pair
};

enum : unsigned { kRowsActive = 1u };

// The window of a lane in a staged row: WIN values from rowp, the float4s that cross a periodic
// seam taken n columns away in the same row, then the centre sums.
template <int R>
__device__ __forceinline__ void rows_window(const float *rowp, const RowsSeg<R> &sg, RowWin<R> &w) {
    using S = RowsSeg<R>;
#pragma unroll
    for (int q = 0; q < S::NQ; ++q) {
        const float4 x = *reinterpret_cast<const float4 *>(rowp + 4 * q + (q == S::QC ? 0 : sg.wd[q]));
        w.v[4 * q + 0] = x.x;
        w.v[4 * q + 1] = x.y;
        w.v[4 * q + 2] = x.z;
        w.v[4 * q + 3] = x.w;
    }
    row_prefix<R>(w);
}

// The update and projection of one output row of a lane (four columns) from its disc sums
// (s01, s23) and centre values uc, and its store (Eq. nonl_CH_nm with beta2 = 0 and the
// projection of Eq. potential_obstacle): sd = fma(-c0, u, S), v = u + fma(c1, sd, c2 u),
// u_new = min(1, max(-1, v)), each packed FP32 pair rounding exactly like the scalar operations.
template <int R>
__device__ __forceinline__ void rows_emit(const RowsSeg<R> &sg, float4 uc, float2 s01, float2 s23) {
    const float2 u01 = make_float2(uc.x, uc.y), u23 = make_float2(uc.z, uc.w);
    const float2 v01 = __fadd2_rn(u01, __ffma2_rn(sg.c1, __ffma2_rn(sg.nc0, u01, s01), __fmul2_rn(sg.c2, u01)));
    const float2 v23 = __fadd2_rn(u23, __ffma2_rn(sg.c1, __ffma2_rn(sg.nc0, u23, s23), __fmul2_rn(sg.c2, u23)));
    *reinterpret_cast<float4 *>(sg.out) =
        make_float4(fminf(1.f, fmaxf(-1.f, v01.x)), fminf(1.f, fmaxf(-1.f, v01.y)), fminf(1.f, fmaxf(-1.f, v23.x)),
                    fminf(1.f, fmaxf(-1.f, v23.y)));
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
__device__ __forceinline__ bool rows_row(RowsAcc<R> &t, const RowsArgs &a, RowsSeg<R> &sg, int q0, RowsShared &sh,
                                         const CUtensorMap *map, const CUtensorMap *map1, float *ring,
                                         uint64_t *bar) {
    using C = RowsCfg<R>;
    const int q = q0 + K;
    t.rp += a.pitch;
    t.cp += a.pitch;
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
        // the copy is issued by lane 0 of warp g mod gw of the group: each warp carries the
        // issue's extra work once every gw chunks, so no warp lags at every barrier
        if (sg.tig == 32 * (g % sg.gw)) {
            // at a segment's first chunk every warp has left the segment before it: its slot
            // takes the segment after the next
            if (q == 0 && sg.kseg > 0) sh.seg[(sg.kseg + 2) % 3] = sh.it.next(a);
            rows_issue<R>(a, sh, map, map1, ring, bar);
        }
    }
    // the centre row q - R enters a new chunk: the stage after the previous centre chunk's
    if ((R % C::CH == 0 ? q % C::CH == 0 : (q - R) % C::CH == 0) && q >= R) {
        t.cst = t.cst + 1 == C::NSTG ? 0 : t.cst + 1;
        t.cp = sg.win0 + t.cst * a.stage_floats + C::R4;
    }
    RowWin<R> win;
    rows_window<R>(t.rp, sg, win);
    rows_classes<R, K>(t, win, std::make_integer_sequence<int, RowsPlan<R>::cls.count>{});
    if (q >= 2 * R) {  // output row q - 2R is complete
        if (opaque_u32(sg.flags) & kRowsActive) {
            constexpr int slot = rows_mod(K - 2 * R, C::S);
            const float4 uc = *reinterpret_cast<const float4 *>(t.cp);  // its centre row, q - R
            rows_emit<R>(sg, uc, t.acc[slot][0], t.acc[slot][1]);
        }
        sg.out += a.t.n;
    }
    return true;
}

template <int R, int... Ks>
__device__ __forceinline__ bool rows_block(RowsAcc<R> &t, const RowsArgs &a, RowsSeg<R> &sg, int q0,
                                           RowsShared &sh, const CUtensorMap *map, const CUtensorMap *map1,
                                           float *ring, uint64_t *bar, int *gfail, std::integer_sequence<int, Ks...>) {
    using C = RowsCfg<R>;
    bool ok = true;
    auto one = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (ok && q0 + K < sg.nrows) {
            ok = rows_row<R, K>(t, a, sg, q0, sh, map, map1, ring, bar);
            if (!ok) *gfail = sg.g0 + (q0 + K) / C::CH;
        }
    };
    (one(std::integral_constant<int, Ks>{}), ...);
    return ok;
}

template <int R>
__global__ void __launch_bounds__(RowsCfg<R>::MAXW * 32, 1)
    step_rows_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map1,
                     const __grid_constant__ RowsArgs a) {
    using C = RowsCfg<R>;
    extern __shared__ __align__(128) float rows_smem[];
    __shared__ __align__(8) uint64_t bars[C::MAXG][C::NSTG];
    __shared__ RowsShared shs[C::MAXG];
    // the next step may be scheduled now; its CTAs take SMs as this step's CTAs leave them
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp groups: a.gs samples x a.strips strips each, independent rings and barriers
    const int gw = a.gs * a.strips, gid = warp / gw, wig = warp - gid * gw;
    const int sl = wig / a.strips, strip = wig - sl * a.strips;  // sample in the group, strip
    // (indexing the shared array itself keeps every ring access a shared-memory load)
    float *ring = rows_smem + gid * C::NSTG * a.stage_floats;
    uint64_t *bar = bars[gid];
    RowsShared &sh = shs[gid];
    const bool leader = (threadIdx.x - 32 * gw * gid) == 0;
    if (leader) {
        for (int i = 0; i < C::NSTG; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.it.init(a, (int)blockIdx.x * a.ng + gid, (int)gridDim.x * a.ng);
        for (int i = 0; i < 3; ++i) sh.seg[i] = sh.it.next(a);
        sh.pslot = 2;  // the first issue advances to slot 0
        sh.pc = sh.pnch = 0;
        sh.pg = 0;
    }
    // the previous step (the producer of the rows read here and the reader of the rows written
    // here) has completed and its stores are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (leader) rows_issue<R>(a, sh, &map, &map1, ring, bar);
    __syncthreads();
    RowsAcc<R> t;
#pragma unroll
    for (int k = 0; k < C::S; ++k) t.acc[k][0] = t.acc[k][1] = make_float2(0.f, 0.f);

    const int n = a.t.n, x = 128 * strip + 4 * lane;
    RowsSeg<R> sg;
    sg.win0 = ring + sl * n + x - C::R4;
#pragma unroll
    for (int q = 0; q < RowsSeg<R>::NQ; ++q) {
        const int c = x / 4 - RowsSeg<R>::QC + q;  // float4 column of the window's q-th float4
        sg.wd[q] = c < 0 ? n : (c >= n / 4 ? -n : 0);
    }
    sg.bid = 1 + gid;
    sg.bthreads = 32 * gw;
    sg.leader = leader;
    sg.tig = threadIdx.x - 32 * gw * gid;
    sg.gw = gw;
    sg.g0 = 0;
    int gfail = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
        // segment k's slot was filled before a barrier that every warp has passed since
        const RowsSegInfo s = sh.seg[k % 3];
        if (s.len == 0) break;
        sg.kseg = k;
        sg.nrows = s.len + 2 * R;
        // the centre row q - R enters chunk 0 at q = R (rows q < R have no centre in use): start
        // one stage before the segment's first chunk
        t.cst = (sg.g0 + C::NSTG - 1) % C::NSTG;
        t.rp = t.cp = sg.win0;
        {
            const int sample = a.gs * s.group + sl;
            const bool active = sample < a.ns && (a.t.steps_ps == nullptr || a.t.step <= a.t.steps_ps[sample]);
            const int smp = active ? sample : 0;
            const StepCoef cf = a.t.coef[smp];
            sg.nc0 = make_float2(-cf.c0, -cf.c0);
            sg.c1 = make_float2(cf.c1, cf.c1);
            sg.c2 = make_float2(cf.c2, cf.c2);
            sg.flags = active ? kRowsActive : 0u;
            sg.out = a.t.dst + (size_t)smp * n * n + (size_t)s.y0 * n + x;
        }
        for (int q0 = 0; ok && q0 < sg.nrows; q0 += C::S)
            ok = rows_block<R>(t, a, sg, q0, sh, &map, &map1, ring, bar, &gfail,
                               std::make_integer_sequence<int, C::S>{});
        sg.g0 += (sg.nrows + C::CH - 1) / C::CH;
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
// sums of four values, then a fixed shuffle tree), read from the fields `plain` when given, else
// from the scratch field that holds each sample's last step: A after an odd number of steps, B
// after an even one (steps_ps: per-sample step counts, or nsteps for all).
__global__ void rows_ooi_kernel(const float *plain, const float *fieldA, const float *fieldB, const int *steps_ps,
                                int nsteps, int n, int strips, size_t ns, double *partials);

// Geometry of the row-streaming kernel for a lattice: samples per CTA, warps, the split of a
// row into k pieces for the tensor map, and the dynamic shared memory.
struct RowsGeom {
    int strips, gs, warps, k, stage_floats;
    size_t smem;
};

struct RowsLauncher {
    int ch, nstg;
    // pdl: launch as a programmatic dependent of the previous kernel in the stream (a step)
    mfmc_status (*fn)(const CUtensorMap &map, const CUtensorMap &map1, const RowsArgs &, int grid, int threads,
                      size_t smem, bool pdl, cudaStream_t);
    int (*blocks_per_sm)(int threads, size_t smem);
};

template <int R>
mfmc_status launch_rows(const CUtensorMap &map, const CUtensorMap &map1, const RowsArgs &a, int grid, int threads,
                        size_t smem, bool pdl, cudaStream_t st) {
    auto kern = step_rows_kernel<R>;
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    MFMC_CUDA(cudaLaunchKernelEx(&cfg, kern, map, map1, a));
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
