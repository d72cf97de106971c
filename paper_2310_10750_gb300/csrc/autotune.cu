// Autotuner: for a model whose algorithm is AUTO, time every candidate disc-sum
// algorithm on a batch large enough to fill the GPU and keep the fastest.  Results are
// cached per (n, R, kernel, boundary, disc) for the life of the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mfmc_internal.h"
#include "tma_step.cuh"

namespace mfmc {

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

mfmc_status autotune(Model &m, cudaStream_t st) {
    if (m.d.beta2 > 0.0) {  // one solver serves beta2 > 0
        m.algo = MFMC_ALGO_ACTIVE_SET;
        m.tuned = 1;
        return MFMC_OK;
    }
    const auto key = std::make_tuple(m.d.n, m.R, (int)m.d.kernel, (int)m.d.bc, m.r2max);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            m.algo = it->second.first;
            if (m.algo == MFMC_ALGO_PREFIX_TMA) m.tma_variant = it->second.second;
            if (m.algo == MFMC_ALGO_ROWS) {
                m.rows_bh = it->second.second / 8;
                m.rows_rx = it->second.second % 8;
            }
            m.tuned = 1;
            return MFMC_OK;
        }
    }
    // candidates: (algorithm, TMA tile variant)
    std::vector<std::pair<int, int>> cands;
    for (int a : {MFMC_ALGO_RESIDENT, MFMC_ALGO_ROWS, MFMC_ALGO_PREFIX_TMA, MFMC_ALGO_PREFIX, MFMC_ALGO_DIRECT,
                  MFMC_ALGO_WEIGHTED, MFMC_ALGO_SPECTRAL}) {
        if (!algo_supported(m, a)) continue;
        if (a == MFMC_ALGO_PREFIX_TMA) {
            for (int v = 0; v < kTmaVariants; ++v) cands.push_back({a, v});
        } else if (a == MFMC_ALGO_ROWS) {
            // second: band height * 8 + columns per thread (band 0: the rows split evenly)
            for (int bh : {0, 64, 128})
                if (bh <= m.d.n && rows_supported(m, 4)) cands.push_back({a, bh * 8 + 4});
        } else {
            cands.push_back({a, 0});
        }
    }
    std::pair<int, int> best = cands.empty() ? std::make_pair((int)MFMC_ALGO_DIRECT, 0) : cands[0];
    if (cands.size() > 1) {
        const size_t nn = (size_t)m.d.n * m.d.n;
        const size_t ns = std::max<size_t>(8, std::min<size_t>(1216, (size_t)(64u << 20) / nn));
        const int steps = std::max(1, std::min(m.d.nsteps, 16));
        float *u0 = nullptr;
        StepCoef *coef = nullptr;
        double *ooi = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        mfmc_status s = MFMC_OK;
        cudaError_t e = cudaMalloc((void **)&u0, ns * nn * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&coef, ns * sizeof(StepCoef));
        if (e == cudaSuccess) e = cudaMalloc((void **)&ooi, ns * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(u0, 0, ns * nn * sizeof(float), st);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) s = cuda_fail(e, "autotune setup");
        if (s == MFMC_OK) s = launch_coefficients(m, nullptr, ns, coef, st);
        float best_ms = 1e30f;
        auto run = [&](std::pair<int, int> c) {
            if (c.first == MFMC_ALGO_PREFIX_TMA)
                return run_solve_tma(m, 0, c.second, coef, u0, ns, steps, nullptr, nullptr, ooi, st);
            if (c.first == MFMC_ALGO_ROWS)
                return run_solve_rows(m, c.second / 8, c.second % 8, coef, u0, ns, steps, nullptr, nullptr, ooi, st);
            return run_solve(m, c.first, coef, u0, ns, steps, nullptr, nullptr, ooi, st);
        };
        for (auto a : cands) {
            if (s != MFMC_OK) break;
            // a candidate that cannot run this model (for example a tile taller than a TMA
            // box allows) is skipped; a failing CUDA call that is not a launch refusal stops
            mfmc_status cs = run(a);  // warm-up
            if (cs != MFMC_OK) {
                (void)cudaGetLastError();
                if (cudaStreamSynchronize(st) != cudaSuccess) {
                    s = cs;
                    break;
                }
                continue;
            }
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && cs == MFMC_OK; ++rep) {
                cudaEventRecord(e0, st);
                cs = run(a);
                cudaEventRecord(e1, st);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    s = cuda_fail(e, "autotune timing");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_min = std::min(ms_min, ms);
            }
            if (s == MFMC_OK && cs == MFMC_OK && ms_min < best_ms) {
                best_ms = ms_min;
                best = a;
            }
        }
        set_error("");
        cudaStreamSynchronize(st);
        cudaFree(u0);
        cudaFree(coef);
        cudaFree(ooi);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s != MFMC_OK) return s;
    }
    m.algo = best.first;
    if (best.first == MFMC_ALGO_PREFIX_TMA) m.tma_variant = best.second;
    if (best.first == MFMC_ALGO_ROWS) {
        m.rows_bh = best.second / 8;
        m.rows_rx = best.second % 8;
    }
    m.tuned = 1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return MFMC_OK;
}

}  // namespace mfmc
