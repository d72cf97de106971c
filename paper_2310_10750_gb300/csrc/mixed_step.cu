// Mixed-fidelity step kernel: one launch advances the samples of up to four models
// (different lattice sizes and horizons R in {2, 4, 8, 16}) by one time step.
//
// The work of a step is one queue of (model, sample, tile) items, ordered heaviest model
// first; persistent CTAs take items from it with an atomic ticket counter, so the cheap
// items of the coarse models fill the SMs while the fine model's items drain.  Each item is
// one TMA box (tile + halo) of that model's ghost-framed field, then the same register-tiled
// prefix-sum computation and fused update as the single-fidelity TMA kernel.  The step loop
// of a batch is captured in a CUDA graph and replayed for repeated batches of the same shape.
// Models whose whole field fits in shared memory (the resident kernel: n <= 128) do not go
// through the queue: each runs all its steps in one resident launch on a second stream,
// concurrently with the step launches, since streaming their tiles through HBM every step
// would cost more than keeping them on chip.
//
// A hierarchy that this queue does not serve but whose every model fits the resident spectral
// form (even n <= 128, any kernel and horizon: the paper's nine models of Section 4) runs as one
// launch of that form over the (model, sample) items of all its models (spectral_resident.cu).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "mfmc_internal.h"
#include "tma_step.cuh"
#include "trace.cuh"

namespace mfmc {

constexpr int kMixGroups = 4;

// Tile shape per R, all with 256 threads: 64 x 64 tiles for R <= 4, 64 x 128 for R = 8,
// 128 x 64 for R = 16.
template <int R>
struct MixShape {
    static constexpr int RY = R <= 4 ? 4 : 8;
    static constexpr int TXT = R <= 8 ? 16 : 32;
    static constexpr int TYT = R <= 8 ? 16 : 8;
};

struct MixedArgs {
    TmaArgs g[kMixGroups];   // per model: outputs, coefficients, partials, step counts, geometry
    int begin[kMixGroups + 1];
    int R[kMixGroups];
    int ngroups, total;
    int *counter;            // ticket counter of this step (zeroed before the solve)
    int *status;
    TraceBuf trace;
};

struct MixedMaps {
    CUtensorMap m[kMixGroups];
};

template <int R>
__device__ __forceinline__ bool mixed_item(const CUtensorMap &map, const TmaArgs &a, int local, float *stage,
                                           uint64_t *bar, uint32_t parity, double *red) {
    using S = MixShape<R>;
    using C = TmaCfg<R, S::RY, S::TXT, S::TYT, 1>;
    const int sample = local / a.tiles, tile = local - sample * a.tiles;
    const int x0 = (tile % a.tiles_x) * C::TX, y0 = (tile / a.tiles_x) * C::TY;
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, C::BOX_BYTES);
        tma_load_3d(stage, &map, bar, x0, y0 + C::R4 - R, sample);
    }
    long long spins = 0;
    bool ok = true;
    while (!mbar_try_wait(bar, parity))
        if (++spins > kWaitLimit) {
            ok = false;
            break;
        }
    if (!__syncthreads_and(ok)) {
        // the copy did not land within the bound: wait for it once more (bounded) so that it
        // does not target the stage after the CTA has gone
        if (threadIdx.x == 0) {
            long long w = 0;
            while (!mbar_try_wait(bar, parity) && ++w < kWaitLimit) {
            }
        }
        return false;
    }
    const bool last = a.last || (a.steps_ps != nullptr && a.step == a.steps_ps[sample]);
    tma_tile_compute<R, S::RY, S::TXT, S::TYT, 1>(stage, a, sample, tile, x0, y0, last, red);
    __syncthreads();  // the stage is free again
    return true;
}

__global__ void __launch_bounds__(256) mixed_step_kernel(const __grid_constant__ MixedMaps maps, MixedArgs a) {
    extern __shared__ unsigned char smem_raw[];
    float *stage = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[8];
    __shared__ int ticket;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t k = 0;  // items loaded by this CTA: the barrier phase
    for (;;) {
        if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = ticket;
        __syncthreads();
        if (item >= a.total) break;
        const unsigned long long t0 = a.trace.rec ? trace_clock() : 0ull;
        int gi = 0;
        while (gi + 1 < a.ngroups && item >= a.begin[gi + 1]) ++gi;
        const TmaArgs &g = a.g[gi];
        const int local = item - a.begin[gi];
        if (g.steps_ps != nullptr && g.step > g.steps_ps[local / g.tiles]) continue;
        bool ok = true;
        switch (a.R[gi]) {
            case 2: ok = mixed_item<2>(maps.m[gi], g, local, stage, &bar, k & 1, red); break;
            case 4: ok = mixed_item<4>(maps.m[gi], g, local, stage, &bar, k & 1, red); break;
            case 8: ok = mixed_item<8>(maps.m[gi], g, local, stage, &bar, k & 1, red); break;
            default: ok = mixed_item<16>(maps.m[gi], g, local, stage, &bar, k & 1, red); break;
        }
        ++k;
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(a.status, 1);
            break;
        }
        if (threadIdx.x == 0) trace_put(a.trace, kTraceMixedStep, (uint32_t)item, (uint32_t)g.step, t0);
    }
}

template <int R>
constexpr size_t mix_stage_bytes() {
    using S = MixShape<R>;
    return (size_t)TmaCfg<R, S::RY, S::TXT, S::TYT, 1>::STAGE_FLOATS * sizeof(float);
}
constexpr size_t kMixSmem =
    std::max(std::max(mix_stage_bytes<2>(), mix_stage_bytes<4>()), std::max(mix_stage_bytes<8>(), mix_stage_bytes<16>())) +
    1024;

struct MixGeom {
    int tx, ty, sw, sh;
};

static bool mix_geom(int R, MixGeom *g) {
    auto set = [&](auto tag) {
        constexpr int RR = decltype(tag)::value;
        using S = MixShape<RR>;
        using C = TmaCfg<RR, S::RY, S::TXT, S::TYT, 1>;
        g->tx = C::TX;
        g->ty = C::TY;
        g->sw = C::SW;
        g->sh = C::SH;
    };
    switch (R) {
        case 2: set(std::integral_constant<int, 2>()); return true;
        case 4: set(std::integral_constant<int, 4>()); return true;
        case 8: set(std::integral_constant<int, 8>()); return true;
        case 16: set(std::integral_constant<int, 16>()); return true;
        default: return false;
    }
}

// Device buffers of one model's samples in a mixed batch (cached between calls).
struct MixGroupBufs {
    size_t cap = 0;
    int n = 0, R = 0;
    bool padded = false;  // ghost-framed buffers and tile partials allocated (step-queue groups)
    float *u0 = nullptr;
    StepCoef *coef = nullptr;
    double *eps = nullptr, *out = nullptr, *theta = nullptr;
    uint64_t *seeds = nullptr;
    int *steps = nullptr;
    TmaBuffers tb;
};

struct MixWorkspace {
    std::mutex mu;
    cudaStream_t st = nullptr;
    cudaStream_t st_res = nullptr;   // resident-kernel groups, concurrent with the step launches
    cudaEvent_t ev_init = nullptr, ev_res = nullptr;
    MixGroupBufs g[kSrMaxModels];
    int *counters = nullptr;
    size_t counters_cap = 0;
    int *status = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<uintptr_t> gkey;
    uint64_t generation = 0;  // bumped by every reallocation: a captured graph holds the old pointers
};

static MixWorkspace &mix_ws() {
    static MixWorkspace *w = new MixWorkspace();  // lives until exit
    return *w;
}

static mfmc_status ensure_group(MixGroupBufs &b, const Model &m, size_t k, bool padded, cudaStream_t st,
                                uint64_t *generation) {
    MixGeom geo{};
    if (padded && !mix_geom(m.R, &geo)) return fail(MFMC_EINVAL, "no mixed-batch tile shape for R = %d", m.R);
    if (b.cap >= k && b.n == m.d.n && b.R == m.R && (b.padded || !padded)) return MFMC_OK;
    ++*generation;
    MFMC_CUDA(cudaStreamSynchronize(st));
    for (void *p : {(void *)b.u0, (void *)b.coef, (void *)b.eps, (void *)b.out, (void *)b.theta, (void *)b.seeds,
                    (void *)b.steps, (void *)b.tb.padA, (void *)b.tb.padB, (void *)b.tb.partials, (void *)b.tb.status})
        cudaFree(p);
    b = MixGroupBufs();
    const int G = (m.R + 3) & ~3, P = m.d.n + 2 * G;
    const size_t nn = (size_t)m.d.n * m.d.n;
    const int tiles = ((m.d.n + geo.tx - 1) / geo.tx) * ((m.d.n + geo.ty - 1) / geo.ty);
    MFMC_CUDA(cudaMalloc((void **)&b.u0, k * nn * sizeof(float)));
    MFMC_CUDA(cudaMalloc((void **)&b.coef, k * sizeof(StepCoef)));
    MFMC_CUDA(cudaMalloc((void **)&b.eps, k * sizeof(double)));
    MFMC_CUDA(cudaMalloc((void **)&b.out, 2 * k * sizeof(double)));
    MFMC_CUDA(cudaMalloc((void **)&b.theta, 12 * k * sizeof(double)));
    MFMC_CUDA(cudaMalloc((void **)&b.seeds, k * sizeof(uint64_t)));
    MFMC_CUDA(cudaMalloc((void **)&b.steps, k * sizeof(int)));
    b.cap = k;
    b.n = m.d.n;
    b.R = m.R;
    if (!padded) return MFMC_OK;
    MFMC_CUDA(cudaMalloc((void **)&b.tb.padA, k * (size_t)P * P * sizeof(float)));
    MFMC_CUDA(cudaMalloc((void **)&b.tb.padB, k * (size_t)P * P * sizeof(float)));
    MFMC_CUDA(cudaMalloc((void **)&b.tb.partials, k * (size_t)tiles * sizeof(double)));
    b.padded = true;
    mfmc_status s = encode_map(&b.tb.mapA, b.tb.padA, P, k, geo.sw, geo.sh);
    if (s == MFMC_OK) s = encode_map(&b.tb.mapB, b.tb.padB, P, k, geo.sw, geo.sh);
    return s;
}

}  // namespace mfmc

using namespace mfmc;

extern "C" mfmc_status mfmc_solve_batch_mixed(mfmc_model *const *models, const mfmc_sample_params *params,
                                              const uint64_t *seeds, size_t ns, double *ooi_out, double *ubar_out) {
    if (ns == 0) return MFMC_OK;
    if (!models || !seeds || !ooi_out) return fail(MFMC_EINVAL, "NULL argument");
    if (ns > (size_t)kMaxNs) return fail(MFMC_EINVAL, "too many samples");
    std::vector<mfmc_model *> order;
    std::map<mfmc_model *, std::vector<size_t>> groups;
    bool tma_route = true, spec_route = true;
    for (size_t i = 0; i < ns; ++i) {
        mfmc_model *m = models[i];
        if (!m) return fail(MFMC_EINVAL, "NULL model at sample %zu", i);
        if (!groups.count(m)) {
            MixGeom geo;
            tma_route = tma_route && m->d.kernel == MFMC_KERNEL_CONSTANT && m->d.bc == MFMC_BC_PERIODIC &&
                        m->integer_R && m->d.beta2 == 0.0 && mix_geom(m->R, &geo);
            spec_route = spec_route && spectral_resident_supported(*m);
            order.push_back(m);
        }
        groups[m].push_back(i);
    }
    tma_route = tma_route && order.size() <= (size_t)kMixGroups;
    spec_route = !tma_route && spec_route && order.size() <= (size_t)kSrMaxModels;
    if (!tma_route && !spec_route)
        return fail(MFMC_EINVAL, "the one-launch mixed batch runs up to %d periodic constant-kernel beta2 = 0 models "
                                 "with R in {2, 4, 8, 16}, or up to %d periodic beta2 = 0 models with even n <= 128 "
                                 "(odd part a product of 3, 5, 7, 11) and 2R + 1 <= n",
                    kMixGroups, kSrMaxModels);
    // heaviest model first in the queue: its items are taken first (the spectral form's cost does
    // not depend on the horizon)
    std::stable_sort(order.begin(), order.end(), [&](mfmc_model *a, mfmc_model *b) {
        const double ra = spec_route ? 1.0 : 2 * a->R + 1, rb = spec_route ? 1.0 : 2 * b->R + 1;
        return (double)a->d.n * a->d.n * ra > (double)b->d.n * b->d.n * rb;
    });
    MixWorkspace &W = mix_ws();
    std::lock_guard<std::mutex> lk(W.mu);
    if (!W.st) {
        MFMC_CUDA(cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking));
        MFMC_CUDA(cudaStreamCreateWithFlags(&W.st_res, cudaStreamNonBlocking));
        MFMC_CUDA(cudaEventCreateWithFlags(&W.ev_init, cudaEventDisableTiming));
        MFMC_CUDA(cudaEventCreateWithFlags(&W.ev_res, cudaEventDisableTiming));
    }
    cudaStream_t st = W.st;
    const int ng = (int)order.size();
    // Models whose whole field fits the shared-memory resident kernel run all their steps
    // there, on a second stream; the others form the step queue of the mixed launches.
    std::vector<char> resident(ng);
    std::vector<int> queue;  // group indices in the step queue, heaviest first
    int max_steps = 0;       // of the queue groups
    std::vector<int> group_steps(ng, 0);
    std::vector<std::vector<int>> steps(ng);
    for (int g = 0; g < ng; ++g) {
        mfmc_model *m = order[g];
        const auto &idx = groups[m];
        resident[g] = spec_route || algo_supported(*m, MFMC_ALGO_RESIDENT) ? 1 : 0;
        if (!resident[g]) queue.push_back(g);
        mfmc_status s = ensure_group(W.g[g], *m, idx.size(), !resident[g], st, &W.generation);
        if (s != MFMC_OK) return s;
        steps[g].resize(idx.size());
        for (size_t q = 0; q < idx.size(); ++q) {
            const mfmc_sample_params *p = params ? &params[idx[q]] : nullptr;
            steps[g][q] = (p && p->nsteps > 0) ? p->nsteps : m->d.nsteps;
            if (steps[g][q] < 1) return fail(MFMC_EINVAL, "the mixed batch needs at least one step per sample");
            group_steps[g] = std::max(group_steps[g], steps[g][q]);
        }
        if (!resident[g]) max_steps = std::max(max_steps, group_steps[g]);
    }
    const int nq = (int)queue.size();
    if ((size_t)std::max(max_steps, 1) > W.counters_cap) {
        MFMC_CUDA(cudaStreamSynchronize(st));
        ++W.generation;
        cudaFree(W.counters);
        W.counters = nullptr;
        MFMC_CUDA(cudaMalloc((void **)&W.counters, std::max(max_steps, 1) * sizeof(int)));
        W.counters_cap = std::max(max_steps, 1);
    }
    if (!W.status) {
        MFMC_CUDA(cudaMalloc((void **)&W.status, sizeof(int)));
        MFMC_CUDA(cudaMemset(W.status, 0, sizeof(int)));
    }
    // inputs: seeds, eps, theta, step counts; initial fields; coefficients; ghost frames
    for (int g = 0; g < ng; ++g) {
        mfmc_model *m = order[g];
        const auto &idx = groups[m];
        const size_t k = idx.size();
        MixGroupBufs &b = W.g[g];
        std::vector<uint64_t> sd(k);
        std::vector<double> ep(k), th(12 * k, 0.0);
        for (size_t q = 0; q < k; ++q) {
            const mfmc_sample_params *p = params ? &params[idx[q]] : nullptr;
            sd[q] = seeds[idx[q]];
            ep[q] = resolve_eps(*m, p, sd[q]);
            resolve_theta(p, sd[q], &th[12 * q]);
        }
        MFMC_CUDA(cudaMemcpyAsync(b.seeds, sd.data(), k * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        MFMC_CUDA(cudaMemcpyAsync(b.eps, ep.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
        MFMC_CUDA(cudaMemcpyAsync(b.theta, th.data(), 12 * k * sizeof(double), cudaMemcpyHostToDevice, st));
        MFMC_CUDA(cudaMemcpyAsync(b.steps, steps[g].data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
        mfmc_status s = launch_init_fields(*m, b.seeds, b.theta, k, b.u0, st);
        if (s == MFMC_OK) s = launch_coefficients(*m, b.eps, k, b.coef, st);
        if (s == MFMC_OK && !resident[g]) s = launch_pad(b.u0, b.tb.padB, m->d.n, (m->R + 3) & ~3, k, st);
        if (s != MFMC_OK) return s;
    }
    // resident groups: one launch each on the second stream, after the inputs are built
    const bool any_resident = nq < ng;
    if (any_resident) {
        MFMC_CUDA(cudaEventRecord(W.ev_init, st));
        MFMC_CUDA(cudaStreamWaitEvent(W.st_res, W.ev_init, 0));
        if (spec_route) {  // every model: one launch over all (model, sample) items
            std::vector<Model *> ms(ng);
            std::vector<SrBatch> bs(ng);
            for (int g = 0; g < ng; ++g) {
                MixGroupBufs &b = W.g[g];
                const size_t k = groups[order[g]].size();
                ms[g] = order[g];
                bs[g].u0 = b.u0;
                bs[g].ubar = b.out + k;
                bs[g].ooi = b.out;
                bs[g].coef = b.coef;
                bs[g].steps_ps = b.steps;
                bs[g].ns = k;
                bs[g].nsteps = group_steps[g];
            }
            mfmc_status s = run_spectral_queue(ms.data(), bs.data(), ng, W.counters, W.st_res);
            if (s != MFMC_OK) return s;
        }
        for (int g = 0; g < ng && !spec_route; ++g) {
            if (!resident[g]) continue;
            MixGroupBufs &b = W.g[g];
            const size_t k = groups[order[g]].size();
            mfmc_status s = run_resident_steps(*order[g], b.coef, b.u0, k, group_steps[g], b.steps, nullptr, b.out + k,
                                               b.out, W.st_res);
            if (s != MFMC_OK) return s;
        }
        MFMC_CUDA(cudaEventRecord(W.ev_res, W.st_res));
    }
    // the step queue: one mixed launch per step, captured once per shape and replayed
    if (nq > 0) {
        std::vector<uintptr_t> key{(uintptr_t)max_steps, (uintptr_t)nq, (uintptr_t)W.generation};
        for (int g : queue) {
            key.push_back((uintptr_t)order[g]);
            key.push_back(groups[order[g]].size());
            key.push_back((uintptr_t)W.g[g].tb.padA);
        }
        key.push_back((uintptr_t)W.counters);
        const TraceBuf trace = trace_buf();  // the captured launches write to the ring of their capture
        key.push_back((uintptr_t)trace.rec);
        if (!(W.gexec && W.gkey == key)) {
            if (W.gexec) cudaGraphExecDestroy(W.gexec);
            W.gexec = nullptr;
            MFMC_CUDA(cudaFuncSetAttribute(mixed_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kMixSmem));
            int dev = 0, sms = 0, per = 0;
            MFMC_CUDA(cudaGetDevice(&dev));
            MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            MFMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mixed_step_kernel, 256, kMixSmem));
            MixedArgs a;
            MixedMaps mp;
            int total = 0;
            for (int qi = 0; qi < nq; ++qi) {
                const int g = queue[qi];
                MixGeom geo{};
                if (!mix_geom(order[g]->R, &geo)) return fail(MFMC_EINVAL, "no mixed-batch tile shape for R = %d", order[g]->R);
                const int n = order[g]->d.n;
                TmaArgs &t = a.g[qi];
                t.dst_plain = nullptr;
                t.coef = W.g[g].coef;
                t.partials = W.g[g].tb.partials;
                t.status = W.status;
                t.steps_ps = W.g[g].steps;
                t.n = n;
                t.P = n + 2 * ((order[g]->R + 3) & ~3);
                t.tiles_x = (n + geo.tx - 1) / geo.tx;
                t.tiles = t.tiles_x * ((n + geo.ty - 1) / geo.ty);
                t.total = (int)groups[order[g]].size() * t.tiles;
                t.last = 0;
                t.periodic = 1;
                a.R[qi] = order[g]->R;
                a.begin[qi] = total;
                total += t.total;
            }
            a.begin[nq] = total;
            a.ngroups = nq;
            a.total = total;
            a.status = W.status;
            a.trace = trace;
            const int grid = std::max(1, std::min(total, sms * std::max(1, per)));
            cudaGraph_t graph = nullptr;
            MFMC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            cudaError_t e = cudaMemsetAsync(W.counters, 0, max_steps * sizeof(int), st);
            for (int k = 1; k <= max_steps && e == cudaSuccess; ++k) {
                for (int qi = 0; qi < nq; ++qi) {
                    const int g = queue[qi];
                    a.g[qi].step = k;
                    a.g[qi].dst = (k & 1) ? W.g[g].tb.padA : W.g[g].tb.padB;
                    mp.m[qi] = (k & 1) ? W.g[g].tb.mapB : W.g[g].tb.mapA;
                }
                a.counter = W.counters + (k - 1);
                mixed_step_kernel<<<grid, 256, kMixSmem, st>>>(mp, a);
                e = cudaGetLastError();
            }
            for (int qi = 0; qi < nq && e == cudaSuccess; ++qi) {
                const int g = queue[qi];
                const size_t k = groups[order[g]].size();
                if (launch_finalize(W.g[g].tb.partials, a.g[qi].tiles, k, order[g]->d.n, W.g[g].out + k, W.g[g].out,
                                    st) != MFMC_OK)
                    e = cudaErrorUnknown;
            }
            cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&W.gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "mixed step graph");
            W.gkey = key;
        }
        MFMC_CUDA(cudaGraphLaunch(W.gexec, st));
    }
    if (any_resident) MFMC_CUDA(cudaStreamWaitEvent(st, W.ev_res, 0));
    std::vector<std::vector<double>> host(ng);
    for (int g = 0; g < ng; ++g) {
        host[g].resize(2 * groups[order[g]].size());
        MFMC_CUDA(cudaMemcpyAsync(host[g].data(), W.g[g].out, host[g].size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  st));
    }
    MFMC_CUDA(cudaStreamSynchronize(st));
    int flag = 0;
    MFMC_CUDA(cudaMemcpy(&flag, W.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        MFMC_CUDA(cudaMemset(W.status, 0, sizeof(int)));
        return fail(MFMC_ETIMEOUT, "a device-side wait gave up");
    }
    for (int g = 0; g < ng; ++g) {
        const auto &idx = groups[order[g]];
        for (size_t q = 0; q < idx.size(); ++q) {
            ooi_out[idx[q]] = host[g][q];
            if (ubar_out) ubar_out[idx[q]] = host[g][idx.size() + q];
        }
    }
    return MFMC_OK;
}
