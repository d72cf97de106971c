// C ABI of the MFMC layer (Section 3): pilot statistics, planning, the estimator and
// the end-to-end run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mfmc_internal.h"

using namespace mfmc;

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

struct StreamGuard {
    cudaStream_t s = nullptr;
    ~StreamGuard() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

mfmc_status stats_to_host(int K, int n, const double *ooi_dev, double *mean, double *sigma, double *rho,
                          cudaStream_t st) {
    DevBuf out;
    MFMC_CUDA(cudaMalloc(&out.p, (size_t)K * 5 * sizeof(double)));
    mfmc_status s = launch_pilot_stats(K, n, ooi_dev, (double *)out.p, st);
    if (s != MFMC_OK) return s;
    std::vector<double> h((size_t)K * 5);
    MFMC_CUDA(cudaMemcpyAsync(h.data(), out.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MFMC_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < K; ++k) {
        if (mean) mean[k] = h[k * 5 + 0];
        if (sigma) sigma[k] = h[k * 5 + 3];
        if (rho) rho[k] = h[k * 5 + 4];
    }
    return MFMC_OK;
}

mfmc_status run_estimate(const mfmc_plan_t *plan, const double *const *ooi_dev, double *est_dev,
                         cudaStream_t st) {
    const int K = plan->K_sel;
    for (int j = 0; j < K; ++j) {
        if (!ooi_dev[j]) return fail(MFMC_EINVAL, "NULL OoI list for model position %d", j);
        if (plan->m[j] < 1) return fail(MFMC_EINVAL, "m_%d < 1", j);
        if (j > 0 && plan->m[j] < plan->m[j - 1]) return fail(MFMC_EINVAL, "sample counts must be nondecreasing");
    }
    // one device block: lists[K] | m[K] | alpha[K] | work[2K + 1]
    const size_t bytes = K * sizeof(double *) + K * sizeof(int64_t) + K * sizeof(double) + (2 * K + 1) * sizeof(double);
    DevBuf blk;
    MFMC_CUDA(cudaMalloc(&blk.p, bytes));
    std::vector<unsigned char> host(bytes);
    std::memcpy(host.data(), ooi_dev, K * sizeof(double *));
    std::memcpy(host.data() + K * sizeof(double *), plan->m, K * sizeof(int64_t));
    std::memcpy(host.data() + K * (sizeof(double *) + sizeof(int64_t)), plan->alpha, K * sizeof(double));
    MFMC_CUDA(cudaMemcpyAsync(blk.p, host.data(), bytes, cudaMemcpyHostToDevice, st));
    unsigned char *b = (unsigned char *)blk.p;
    double *work = (double *)(b + K * (sizeof(double *) + sizeof(int64_t) + sizeof(double)));
    mfmc_status s = launch_estimate(K, (const double *const *)b, (const int64_t *)(b + K * sizeof(double *)),
                                    (const double *)(b + K * (sizeof(double *) + sizeof(int64_t))), work, st);
    if (s != MFMC_OK) return s;
    MFMC_CUDA(cudaMemcpyAsync(est_dev, work + 2 * K, sizeof(double), cudaMemcpyDeviceToDevice, st));
    // the block is freed on return: wait for the kernels that read it
    MFMC_CUDA(cudaStreamSynchronize(st));
    return MFMC_OK;
}

// Solve `count` samples of one model with seeds seed0 .. seed0+count-1, OoIs to ooi_dev.
mfmc_status solve_seeds(mfmc_model *m, uint64_t seed0, size_t count, double *ooi_dev, cudaStream_t st) {
    const size_t nn = (size_t)m->d.n * m->d.n;
    const size_t chunk = std::max<size_t>(1, std::min<size_t>(count, (size_t)(1ull << 30) / (nn * sizeof(float))));
    DevBuf u0, eps;
    MFMC_CUDA(cudaMalloc(&u0.p, chunk * nn * sizeof(float)));
    MFMC_CUDA(cudaMalloc(&eps.p, chunk * sizeof(double)));
    std::vector<uint64_t> seeds(chunk);
    std::vector<double> ep(chunk);
    for (size_t o = 0; o < count; o += chunk) {
        const size_t k = std::min(chunk, count - o);
        for (size_t q = 0; q < k; ++q) {
            seeds[q] = seed0 + o + q;
            ep[q] = resolve_eps(*m, nullptr, seeds[q]);
        }
        MFMC_CUDA(cudaMemcpyAsync(eps.p, ep.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
        mfmc_status s = mfmc_init_fields(m, nullptr, seeds.data(), k, (float *)u0.p, st);
        if (s != MFMC_OK) return s;
        s = mfmc_solve_fields(m, (const double *)eps.p, (const float *)u0.p, k, nullptr, nullptr, ooi_dev + o, st);
        if (s != MFMC_OK) return s;
        MFMC_CUDA(cudaStreamSynchronize(st));
    }
    return MFMC_OK;
}

}  // namespace

extern "C" {

mfmc_status mfmc_pilot_stats(int K, int n, const double *ooi_dev, double *mean, double *sigma, double *rho,
                             void *stream) {
    if (K < 1 || K > MFMC_MAX_MODELS || n < 2 || !ooi_dev) return fail(MFMC_EINVAL, "invalid pilot statistics arguments");
    return stats_to_host(K, n, ooi_dev, mean, sigma, rho, (cudaStream_t)stream);
}

mfmc_status mfmc_plan(int K, int n_pilot, const double *pilot_ooi, const double *costs, double budget, int policy,
                      const int *explicit_idx, int explicit_len, mfmc_plan_t *out) {
    if (K < 1 || K > MFMC_MAX_MODELS || n_pilot < 2 || !pilot_ooi || !costs || !out)
        return fail(MFMC_EINVAL, "invalid plan arguments");
    StreamGuard sg;
    MFMC_CUDA(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
    DevBuf d;
    const size_t bytes = (size_t)K * n_pilot * sizeof(double);
    MFMC_CUDA(cudaMalloc(&d.p, bytes));
    MFMC_CUDA(cudaMemcpyAsync(d.p, pilot_ooi, bytes, cudaMemcpyHostToDevice, sg.s));
    std::vector<double> mean(K), sigma(K), rho(K);
    mfmc_status s = stats_to_host(K, n_pilot, (const double *)d.p, mean.data(), sigma.data(), rho.data(), sg.s);
    if (s != MFMC_OK) return s;
    return plan_from_stats(K, mean.data(), sigma.data(), rho.data(), costs, budget, policy, explicit_idx, explicit_len,
                           out);
}

mfmc_status mfmc_plan_from_stats(int K, const double *rho, const double *sigma, const double *costs, double budget,
                                 int policy, const int *explicit_idx, int explicit_len, mfmc_plan_t *out) {
    if (K < 1 || K > MFMC_MAX_MODELS || !rho || !sigma || !costs || !out)
        return fail(MFMC_EINVAL, "invalid plan arguments");
    for (int k = 0; k < K; ++k) {
        if (!std::isfinite(rho[k]) || std::fabs(rho[k]) > 1.0) return fail(MFMC_EINVAL, "rho of model %d outside [-1, 1]", k);
        if (!std::isfinite(sigma[k]) || !(sigma[k] > 0)) return fail(MFMC_EINVAL, "sigma of model %d must be > 0", k);
        if (!std::isfinite(costs[k])) return fail(MFMC_EINVAL, "cost of model %d is not finite", k);
    }
    if (!std::isfinite(budget)) return fail(MFMC_EINVAL, "budget is not finite");
    const std::vector<double> mean(K, 0.0);
    return plan_from_stats(K, mean.data(), sigma, rho, costs, budget, policy, explicit_idx, explicit_len, out);
}

mfmc_status mfmc_estimate_device(const mfmc_plan_t *plan, const double *const *ooi_dev, double *estimate_dev,
                                 void *stream) {
    if (!plan || !ooi_dev || !estimate_dev || plan->K_sel < 1 || plan->K_sel > MFMC_MAX_MODELS)
        return fail(MFMC_EINVAL, "invalid estimate arguments");
    return run_estimate(plan, ooi_dev, estimate_dev, (cudaStream_t)stream);
}

mfmc_status mfmc_estimate(const mfmc_plan_t *plan, const double *const *ooi, double *estimate) {
    if (!plan || !ooi || !estimate || plan->K_sel < 1 || plan->K_sel > MFMC_MAX_MODELS)
        return fail(MFMC_EINVAL, "invalid estimate arguments");
    const int K = plan->K_sel;
    StreamGuard sg;
    MFMC_CUDA(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
    std::vector<DevBuf> bufs(K);
    std::vector<const double *> ptrs(K);
    for (int j = 0; j < K; ++j) {
        if (!ooi[j] || plan->m[j] < 1) return fail(MFMC_EINVAL, "invalid OoI list %d", j);
        const size_t bytes = (size_t)plan->m[j] * sizeof(double);
        MFMC_CUDA(cudaMalloc(&bufs[j].p, bytes));
        MFMC_CUDA(cudaMemcpyAsync(bufs[j].p, ooi[j], bytes, cudaMemcpyHostToDevice, sg.s));
        ptrs[j] = (const double *)bufs[j].p;
    }
    DevBuf est;
    MFMC_CUDA(cudaMalloc(&est.p, sizeof(double)));
    mfmc_status s = run_estimate(plan, ptrs.data(), (double *)est.p, sg.s);
    if (s != MFMC_OK) return s;
    MFMC_CUDA(cudaMemcpyAsync(estimate, est.p, sizeof(double), cudaMemcpyDeviceToHost, sg.s));
    MFMC_CUDA(cudaStreamSynchronize(sg.s));
    return MFMC_OK;
}

mfmc_status mfmc_run(mfmc_model *const *models, int K, int n_pilot, double budget, int policy, uint64_t seed_base,
                     const double *costs, mfmc_plan_t *plan_out, double *estimate) {
    if (!models || K < 1 || K > MFMC_MAX_MODELS || n_pilot < 2 || !plan_out || !estimate || !(budget > 0))
        return fail(MFMC_EINVAL, "invalid run arguments");
    if (policy == 3) return fail(MFMC_EINVAL, "policy 3 needs mfmc_plan with an explicit subset");
    for (int k = 0; k < K; ++k)
        if (!models[k]) return fail(MFMC_EINVAL, "NULL model %d", k);
    StreamGuard sg;
    MFMC_CUDA(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
    // pilot: every model on the same n_pilot seeds
    DevBuf pilot;
    MFMC_CUDA(cudaMalloc(&pilot.p, (size_t)K * n_pilot * sizeof(double)));
    std::vector<double> measured(K);
    cudaEvent_t e0, e1;
    MFMC_CUDA(cudaEventCreate(&e0));
    MFMC_CUDA(cudaEventCreate(&e1));
    mfmc_status s = MFMC_OK;
    for (int k = 0; k < K && s == MFMC_OK; ++k) {
        // warm the model (autotuning, scratch) outside the cost measurement
        s = solve_seeds(models[k], seed_base, std::min(n_pilot, 2), (double *)pilot.p + (size_t)k * n_pilot, sg.s);
        if (s != MFMC_OK) break;
        cudaEventRecord(e0, sg.s);
        s = solve_seeds(models[k], seed_base, n_pilot, (double *)pilot.p + (size_t)k * n_pilot, sg.s);
        cudaEventRecord(e1, sg.s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        measured[k] = (double)ms * 1e-3 / n_pilot;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MFMC_OK) return s;
    std::vector<double> mean(K), sigma(K), rho(K);
    s = stats_to_host(K, n_pilot, (const double *)pilot.p, mean.data(), sigma.data(), rho.data(), sg.s);
    if (s != MFMC_OK) return s;
    s = plan_from_stats(K, mean.data(), sigma.data(), rho.data(), costs ? costs : measured.data(), budget, policy,
                        nullptr, 0, plan_out);
    if (s != MFMC_OK) return s;
    // estimation: model i_j on the first m_j estimation seeds (disjoint from the pilot)
    const int Ks = plan_out->K_sel;
    std::vector<DevBuf> lists(Ks);
    std::vector<const double *> ptrs(Ks);
    for (int j = 0; j < Ks; ++j) {
        const size_t mj = (size_t)plan_out->m[j];
        MFMC_CUDA(cudaMalloc(&lists[j].p, std::max<size_t>(1, mj) * sizeof(double)));
        s = solve_seeds(models[plan_out->idx[j]], seed_base + (uint64_t)n_pilot, mj, (double *)lists[j].p, sg.s);
        if (s != MFMC_OK) return s;
        ptrs[j] = (const double *)lists[j].p;
    }
    DevBuf est;
    MFMC_CUDA(cudaMalloc(&est.p, sizeof(double)));
    s = run_estimate(plan_out, ptrs.data(), (double *)est.p, sg.s);
    if (s != MFMC_OK) return s;
    MFMC_CUDA(cudaMemcpyAsync(estimate, est.p, sizeof(double), cudaMemcpyDeviceToHost, sg.s));
    MFMC_CUDA(cudaStreamSynchronize(sg.s));
    return MFMC_OK;
}

}  // extern "C"
