// Host side of the resident spectral queue (spectral_queue.cuh): one launch over the samples of up
// to kSrMaxModels periodic beta2 = 0 models on small lattices (n <= 128), for one model
// (MFMC_ALGO_SPECTRAL on an n other than 64, 128 and 1024) or a hierarchy (the mixed batch).
//
// The work is a queue of (model, sample group) items, heaviest model first.  Persistent CTAs take
// items with an atomic ticket counter; an item is a whole solve kept in shared memory for every
// step: on n = 128 (one sample) and n = 64 (four samples) by the register-transform form, on any
// other even n whose odd part is a product of 3, 5, 7 and 11 by the mixed-radix transforms of
// smem_fft.cuh (the paper's n = 88 on its compile-time plan), each step's disc sums going straight
// into the update of Eq. (nonl_CH_nm) with beta2 = 0 and the projection of Eq.
// (potential_obstacle).  So the samples of every fidelity of the paper's hierarchy (Section 4:
// h in {1/128, 1/88, 1/64}, any horizon, the Gaussian kernel, delta/h = 16.5 included) run
// together in one launch, and the cheap items of the coarse models fill the SMs while the fine
// model's items drain.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mfmc_internal.h"
#include "spectral_queue.cuh"

namespace mfmc {

bool spectral_resident_supported(const Model &m) {
    FftPlan p;
    return m.d.bc == MFMC_BC_PERIODIC && m.d.beta2 == 0.0 && m.d.n <= kFftMaxN && m.d.n % 2 == 0 &&
           2 * m.R + 1 <= m.d.n && fft_plan(m.d.n, &p);
}

// The mixed-radix form's tables: K^ / n^2 in FP32 at [ky][n/2 + 1] (from the same FP32 weights as
// the other FP32 kernels, summed in FP64) and W_n^j.
static mfmc_status sr_tables(Model &m) {
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    if (m.d_khat32 && m.sr_dev == dev) return MFMC_OK;
    cudaFree(m.d_khat32);
    cudaFree(m.d_tw32);
    m.d_khat32 = nullptr;
    m.d_tw32 = nullptr;
    const int n = m.d.n, nh = n / 2 + 1;
    const std::vector<float> kt = spectral_khat(m, n);  // [kx][ky]
    std::vector<float> kh((size_t)n * nh);
    for (int ky = 0; ky < n; ++ky)
        for (int kx = 0; kx < nh; ++kx) kh[(size_t)ky * nh + kx] = kt[(size_t)kx * n + ky];
    std::vector<float2> tw(n);
    for (int j = 0; j < n; ++j)
        tw[j] = make_float2((float)std::cos(2.0 * M_PI * j / n), (float)-std::sin(2.0 * M_PI * j / n));
    MFMC_CUDA(cudaMalloc((void **)&m.d_khat32, kh.size() * sizeof(float)));
    MFMC_CUDA(cudaMemcpy(m.d_khat32, kh.data(), kh.size() * sizeof(float), cudaMemcpyHostToDevice));
    MFMC_CUDA(cudaMalloc((void **)&m.d_tw32, tw.size() * sizeof(float2)));
    MFMC_CUDA(cudaMemcpy(m.d_tw32, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    m.sr_dev = dev;
    return MFMC_OK;
}

mfmc_status run_spectral_queue(Model *const *models, const SrBatch *batches, int nm, int *counter, cudaStream_t st) {
    if (nm < 1 || nm > kSrMaxModels) return fail(MFMC_EINVAL, "1 to %d models per resident spectral launch", kSrMaxModels);
    SqArgs a{};
    size_t smem = 0;
    long long total = 0;
    bool small = false;
    for (int k = 0; k < nm; ++k) {
        Model &m = *models[k];
        if (!spectral_resident_supported(m))
            return fail(MFMC_EINVAL, "the resident spectral form needs a periodic beta2 = 0 model with an even n <= 128 "
                                     "whose odd part factors into 3, 5, 7 and 11, and 2R + 1 <= n");
        const SrBatch &b = batches[k];
        SqModelDev &d = a.m[k];
        const int n = m.d.n;
        d.kind = n == 128 ? kSqSmall128 : (n == 64 ? kSqSmall64 : kSqGeneric);
        d.spc = d.kind == kSqSmall64 ? 4 : 1;
        small = small || d.kind != kSqGeneric;
        if (d.kind == kSqGeneric) {
            mfmc_status s = sr_tables(m);
            if (s != MFMC_OK) return s;
            d.khat = m.d_khat32;
            d.tw = m.d_tw32;
        } else {
            mfmc_status s = spectral_small_tables(m, &d.khat, &d.tw);
            if (s != MFMC_OK) return s;
        }
        d.u0 = b.u0;
        d.uT = b.uT;
        d.ubar = b.ubar;
        d.ooi = b.ooi;
        d.coef = b.coef;
        d.steps_ps = b.steps_ps;
        fft_plan(n, &d.plan);
        d.ns = (int)std::min<size_t>(b.ns, (size_t)INT32_MAX);
        d.nsteps = b.nsteps;
        a.begin[k] = (int)total;
        total += (long long)((b.ns + d.spc - 1) / d.spc);
        if (b.ns > (size_t)INT32_MAX / 2 || total > INT32_MAX / 2)
            return fail(MFMC_EINVAL, "batch too large for the resident spectral form");
        smem = std::max(smem, spectral_queue_smem(d.kind, n));
    }
    a.begin[nm] = (int)total;
    a.nm = nm;
    a.total = (int)total;
    if (total == 0) return MFMC_OK;
    int dev = 0, sms = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MFMC_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    a.counter = counter;
    a.trace = trace_buf();
    const int per = spectral_queue_blocks_per_sm(small, smem);
    const int grid = (int)std::min<long long>(total, (long long)sms * per);
    return launch_spectral_queue(small, a, grid, smem, st);
}

mfmc_status run_solve_spectral_resident(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                                        float *uT, double *ubar, double *ooi, cudaStream_t st) {
    Model *mp = &m;
    SrBatch b;
    b.u0 = u0;
    b.uT = uT;
    b.ubar = ubar;
    b.ooi = ooi;
    b.coef = coef;
    b.steps_ps = nullptr;
    b.ns = ns;
    b.nsteps = nsteps;
    if (!m.sr_counter) MFMC_CUDA(cudaMalloc((void **)&m.sr_counter, sizeof(int)));
    return run_spectral_queue(&mp, &b, 1, m.sr_counter, st);
}

}  // namespace mfmc
