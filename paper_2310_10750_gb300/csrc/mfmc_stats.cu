// FP64 cross-sample statistics (Section 3.1) and the telescoping MFMC estimator
// (Eq. MFMC_estimator) on the GPU.  All reductions use a fixed order: thread t adds the
// elements t, t + 256, ... in order, then thread 0 adds the 256 partials in order.
#include <cuda_runtime.h>

#include "mfmc_internal.h"

namespace mfmc {

constexpr int ST_NT = 256;

__device__ double fixed_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < ST_NT; ++i) t += red[i];
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

// One CTA per model k: mean_k, variance_k (n-1), Cov(f_1, f_k) (n-1), sigma_k and rho_1k.
// out[k * 5 + {0..4}] = mean, var, cov1k, sigma, rho.
__global__ void __launch_bounds__(ST_NT) pilot_stats_kernel(int n, const double *ooi, double *out) {
    __shared__ double red[ST_NT];
    const int k = blockIdx.x;
    const double *f1 = ooi;
    const double *fk = ooi + (size_t)k * n;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += ST_NT) {
        a += f1[i];
        b += fk[i];
    }
    const double m1 = fixed_sum(a, red) / n;
    const double mk = fixed_sum(b, red) / n;
    double v1 = 0.0, vk = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += ST_NT) {
        const double d1 = f1[i] - m1, dk = fk[i] - mk;
        v1 += d1 * d1;
        vk += dk * dk;
        c += d1 * dk;
    }
    const double var1 = fixed_sum(v1, red) / (n - 1);
    const double vark = fixed_sum(vk, red) / (n - 1);
    const double cov = fixed_sum(c, red) / (n - 1);
    if (threadIdx.x == 0) {
        const double s1 = sqrt(var1), sk = sqrt(vark);
        out[k * 5 + 0] = mk;
        out[k * 5 + 1] = vark;
        out[k * 5 + 2] = cov;
        out[k * 5 + 3] = sk;
        out[k * 5 + 4] = (k == 0) ? 1.0 : cov / (s1 * sk);
    }
}

mfmc_status launch_pilot_stats(int K, int n, const double *ooi, double *out_dev, cudaStream_t st) {
    pilot_stats_kernel<<<K, ST_NT, 0, st>>>(n, ooi, out_dev);
    MFMC_LAUNCHED("mfmc_stats launch 1");
    return MFMC_OK;
}

// One CTA per selected model j: means of the first m_j and of the first m_{j-1} values.
__global__ void __launch_bounds__(ST_NT) prefix_means_kernel(const double *const *lists, const int64_t *m,
                                                             double *means) {
    __shared__ double red[ST_NT];
    const int j = blockIdx.x;
    const double *f = lists[j];
    const int64_t mj = m[j], mp = j > 0 ? m[j - 1] : 0;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < mj; i += ST_NT) a += f[i];
    for (int64_t i = threadIdx.x; i < mp; i += ST_NT) b += f[i];
    const double sa = fixed_sum(a, red);
    const double sb = fixed_sum(b, red);
    if (threadIdx.x == 0) {
        means[2 * j] = sa / (double)mj;
        means[2 * j + 1] = mp > 0 ? sb / (double)mp : 0.0;
    }
}

// Q = Q^{(i_1)}_{m_1} + sum_{j>=2} alpha_j (Q^{(i_j)}_{m_j} - Q^{(i_j)}_{m_{j-1}}), in j order.
__global__ void combine_kernel(int K, const double *means, const double *alpha, double *est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double q = means[0];
    for (int j = 1; j < K; ++j) q += alpha[j] * (means[2 * j] - means[2 * j + 1]);
    *est = q;
}

mfmc_status launch_estimate(int K, const double *const *lists_dev, const int64_t *m_dev, const double *alpha_dev,
                            double *work_dev, cudaStream_t st) {
    // work_dev: 2K means followed by the estimate
    prefix_means_kernel<<<K, ST_NT, 0, st>>>(lists_dev, m_dev, work_dev);
    combine_kernel<<<1, 32, 0, st>>>(K, work_dev, alpha_dev, work_dev + 2 * K);
    MFMC_LAUNCHED("mfmc_stats launch 2");
    return MFMC_OK;
}

}  // namespace mfmc
