// Spectral form of the disc sum (MFMC_ALGO_FFT): on the periodic lattice the nodal
// quadrature (gamma * u)_i = sum_{z in D} w_z u_{i+z} is a circular convolution, so
//   S = IFFT( FFT(u) * FFT(K) ),   K[z mod n] = w_z on the disc,
// whose cost does not depend on the horizon.  The transforms are cuFFT's (a library, loaded
// at run time: this path is a comparison point for very large horizons, not the
// register-tiled kernels' hot path); the spectrum of K is formed once per model and batch
// shape, the product and the fused update (the same update as every other kernel) are this
// file's kernels.  Periodic boundary only; any radial kernel and any radius delta/h.
#include <cuda_runtime.h>
#include <cufft.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "mfmc_internal.h"

namespace mfmc {

// cuFFT entry points, resolved from the shared library on first use.
struct CufftApi {
    bool ok = false;
    cufftResult (*plan_many)(cufftHandle *, int, int *, int *, int, int, int *, int, int, cufftType, int) = nullptr;
    cufftResult (*exec_r2c)(cufftHandle, cufftReal *, cufftComplex *) = nullptr;
    cufftResult (*exec_c2r)(cufftHandle, cufftComplex *, cufftReal *) = nullptr;
    cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal *, cufftDoubleComplex *) = nullptr;
    cufftResult (*exec_z2d)(cufftHandle, cufftDoubleComplex *, cufftDoubleReal *) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
};

static const CufftApi &cufft_api() {
    static CufftApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = dlopen("libcufft.so.12", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("libcufft.so", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        api.plan_many = reinterpret_cast<decltype(api.plan_many)>(dlsym(h, "cufftPlanMany"));
        api.exec_r2c = reinterpret_cast<decltype(api.exec_r2c)>(dlsym(h, "cufftExecR2C"));
        api.exec_c2r = reinterpret_cast<decltype(api.exec_c2r)>(dlsym(h, "cufftExecC2R"));
        api.set_stream = reinterpret_cast<decltype(api.set_stream)>(dlsym(h, "cufftSetStream"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "cufftDestroy"));
        api.exec_d2z = reinterpret_cast<decltype(api.exec_d2z)>(dlsym(h, "cufftExecD2Z"));
        api.exec_z2d = reinterpret_cast<decltype(api.exec_z2d)>(dlsym(h, "cufftExecZ2D"));
        api.ok = api.plan_many && api.exec_r2c && api.exec_c2r && api.set_stream && api.destroy;
    });
    return api;
}

bool fft_available() { return cufft_api().ok; }
bool fft64_available() { return cufft_api().ok && cufft_api().exec_d2z && cufft_api().exec_z2d; }

// Per-model state: plans for the last batch size, the spectrum of K and the buffers.
struct FftState {
    int n = 0;
    size_t batch = 0;
    cufftHandle fwd = 0, inv = 0, one = 0;
    bool have_plans = false, have_one = false;
    cufftComplex *khat = nullptr;  // FFT(K), [n][n/2 + 1]
    cufftComplex *spec = nullptr;  // [batch][n][n/2 + 1]
    float *S = nullptr;            // disc sums, [batch][n][n]
    float *bufA = nullptr, *bufB = nullptr;
};

void fft_release(FftState *f) {
    if (!f) return;
    const CufftApi &api = cufft_api();
    if (f->have_plans && api.ok) {
        api.destroy(f->fwd);
        api.destroy(f->inv);
    }
    if (f->have_one && api.ok) api.destroy(f->one);
    cudaFree(f->khat);
    cudaFree(f->spec);
    cudaFree(f->S);
    cudaFree(f->bufA);
    cudaFree(f->bufB);
    delete f;
}

// spec[b][k] *= khat[k] / n^2 (the inverse transform is unnormalised)
__global__ void fft_multiply_kernel(cufftComplex *spec, const cufftComplex *khat, size_t per, size_t total,
                                    float inv_nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const cufftComplex a = spec[i], k = khat[i % per];
        spec[i] = make_cuFloatComplex((a.x * k.x - a.y * k.y) * inv_nn, (a.x * k.y + a.y * k.x) * inv_nn);
    }
}

// The update of every kernel here: v = u + c1 (S - c0 u) + c2 u, projected onto [-1, 1].
__global__ void fft_update_kernel(const float *u, const float *S, float *dst, const StepCoef *coef, size_t nn4,
                                  size_t total4) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const StepCoef cf = coef[i / nn4];
        const float4 uc = reinterpret_cast<const float4 *>(u)[i];
        const float4 s = reinterpret_cast<const float4 *>(S)[i];
        const float ui[4] = {uc.x, uc.y, uc.z, uc.w}, si[4] = {s.x, s.y, s.z, s.w};
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float sd = fmaf(-cf.c0, ui[k], si[k]);
            const float v = ui[k] + fmaf(cf.c1, sd, cf.c2 * ui[k]);
            o[k] = fminf(1.f, fmaxf(-1.f, v));
        }
        reinterpret_cast<float4 *>(dst)[i] = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// Per-sample FP64 sum of a field in a fixed order (thread t adds t, t + 256, ...; then the
// 256 partials in order), and the OoI from it.
__global__ void __launch_bounds__(256) fft_ooi_kernel(const float *u, size_t nn, double *ubar, double *ooi) {
    __shared__ double red[256];
    const float *f = u + blockIdx.x * nn;
    double t = 0.0;
    for (size_t i = threadIdx.x; i < nn; i += 256) t += (double)f[i];
    red[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 256; ++i) s += red[i];
        const double mean = s / (double)nn;
        if (ubar) ubar[blockIdx.x] = mean;
        if (ooi) ooi[blockIdx.x] = 0.5 * (1.0 + mean);
    }
}


#define MFMC_CUFFT(call)                                                          \
    do {                                                                          \
        cufftResult r_ = (call);                                                  \
        if (r_ != CUFFT_SUCCESS) return fail(MFMC_ECUDA, "%s failed (%d)", #call, (int)r_); \
    } while (0)

// Plans for `ns` samples, the spectrum of the disc weights, and buffers.
static mfmc_status fft_prepare(Model &m, size_t ns, cudaStream_t st) {
    const CufftApi &api = cufft_api();
    if (!api.ok) return fail(MFMC_ECUDA, "cuFFT (libcufft.so) could not be loaded: the FFT path is unavailable");
    if (!m.fft) m.fft = new FftState();
    FftState &f = *m.fft;
    const int n = m.d.n;
    const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
    if (f.n != n || !f.have_one) {
        // the spectrum of K, once per model
        if (f.have_one) api.destroy(f.one);
        f.have_one = false;
        int dims[2] = {n, n};
        MFMC_CUFFT(api.plan_many(&f.one, 2, dims, nullptr, 1, (int)nn, nullptr, 1, (int)nh, CUFFT_R2C, 1));
        f.have_one = true;
        std::vector<float> K(nn, 0.f);
        for (int dy = -m.R; dy <= m.R; ++dy) {
            const int w = m.widths[dy < 0 ? -dy : dy];
            for (int dx = -w; dx <= w; ++dx) {
                const float wt = m.d.kernel == MFMC_KERNEL_CONSTANT ? 1.f : m.wtab[dx * dx + dy * dy];
                K[(size_t)((dy + n) % n) * n + (dx + n) % n] = wt;  // 2R + 1 <= n: no two points share a cell
            }
        }
        float *Kd = nullptr;
        cudaFree(f.khat);
        f.khat = nullptr;
        MFMC_CUDA(cudaMalloc((void **)&Kd, nn * sizeof(float)));
        MFMC_CUDA(cudaMalloc((void **)&f.khat, nh * sizeof(cufftComplex)));
        MFMC_CUDA(cudaMemcpy(Kd, K.data(), nn * sizeof(float), cudaMemcpyHostToDevice));
        MFMC_CUFFT(api.set_stream(f.one, st));
        cufftResult r = api.exec_r2c(f.one, Kd, f.khat);
        MFMC_CUDA(cudaStreamSynchronize(st));
        cudaFree(Kd);
        if (r != CUFFT_SUCCESS) return fail(MFMC_ECUDA, "cuFFT transform of the disc weights failed (%d)", (int)r);
        f.n = n;
        f.batch = 0;
    }
    if (f.batch != ns || !f.have_plans) {
        MFMC_CUDA(cudaStreamSynchronize(st));
        if (f.have_plans) {
            api.destroy(f.fwd);
            api.destroy(f.inv);
        }
        f.have_plans = false;
        for (void *p : {(void *)f.spec, (void *)f.S, (void *)f.bufA, (void *)f.bufB}) cudaFree(p);
        f.spec = nullptr;
        f.S = f.bufA = f.bufB = nullptr;
        int dims[2] = {n, n};
        MFMC_CUFFT(api.plan_many(&f.fwd, 2, dims, nullptr, 1, (int)nn, nullptr, 1, (int)nh, CUFFT_R2C, (int)ns));
        cufftResult r = api.plan_many(&f.inv, 2, dims, nullptr, 1, (int)nh, nullptr, 1, (int)nn, CUFFT_C2R, (int)ns);
        if (r != CUFFT_SUCCESS) {
            api.destroy(f.fwd);
            return fail(MFMC_ECUDA, "cufftPlanMany (inverse) failed (%d)", (int)r);
        }
        f.have_plans = true;
        MFMC_CUDA(cudaMalloc((void **)&f.spec, ns * nh * sizeof(cufftComplex)));
        MFMC_CUDA(cudaMalloc((void **)&f.S, ns * nn * sizeof(float)));
        MFMC_CUDA(cudaMalloc((void **)&f.bufA, ns * nn * sizeof(float)));
        MFMC_CUDA(cudaMalloc((void **)&f.bufB, ns * nn * sizeof(float)));
        f.batch = ns;
    }
    MFMC_CUFFT(api.set_stream(f.fwd, st));
    MFMC_CUFFT(api.set_stream(f.inv, st));
    return MFMC_OK;
}

mfmc_status run_solve_fft(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps, float *uT,
                          double *ubar, double *ooi, cudaStream_t st) {
    if (m.d.bc != MFMC_BC_PERIODIC) return fail(MFMC_EINVAL, "the FFT path is periodic only");
    if (ns > (size_t)(1 << 30) / ((size_t)m.d.n * m.d.n)) return fail(MFMC_EINVAL, "batch too large for the FFT path");
    mfmc_status s = fft_prepare(m, ns, st);
    if (s != MFMC_OK) return s;
    const CufftApi &api = cufft_api();
    FftState &f = *m.fft;
    const int n = m.d.n;
    const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
    const float *src = u0;
    for (int k = 1; k <= nsteps; ++k) {
        float *dst = (k == nsteps && uT) ? uT : ((k & 1) ? f.bufA : f.bufB);
        // cuFFT's R2C input is non-const in its signature; it does not write it
        MFMC_CUFFT(api.exec_r2c(f.fwd, const_cast<float *>(src), f.spec));
        const size_t tot = ns * nh;
        fft_multiply_kernel<<<(unsigned)std::min<size_t>((tot + 255) / 256, 152 * 64), 256, 0, st>>>(
            f.spec, f.khat, nh, tot, 1.f / (float)nn);
        MFMC_LAUNCHED("fft_solver launch 1");
        MFMC_CUFFT(api.exec_c2r(f.inv, f.spec, f.S));
        const size_t tot4 = ns * nn / 4;
        fft_update_kernel<<<(unsigned)std::min<size_t>((tot4 + 255) / 256, 152 * 64), 256, 0, st>>>(
            src, f.S, dst, coef, nn / 4, tot4);
        MFMC_LAUNCHED("fft_solver launch 2");
        src = dst;
    }
    for (size_t o = 0; o < ns; o += 65535) {
        const unsigned g = (unsigned)std::min<size_t>(65535, ns - o);
        fft_ooi_kernel<<<g, 256, 0, st>>>(src + o * nn, nn, ubar ? ubar + o : nullptr, ooi ? ooi + o : nullptr);
    }
    MFMC_LAUNCHED("fft_solver launch 3");
    return MFMC_OK;
}

// ---- FP64 disc sums for the beta2 > 0 solver ----------------------------------------------
// S_i = sum_{z in D} w_z u_{i+z} for a batch of FP64 fields held in strided per-sample blocks,
// as IFFT(FFT(u) * Khat), through cuFFT: the lattices whose half spectrum does not fit in a
// CTA's shared memory (n > 128; the solver transforms smaller ones itself).  The weights are radial, hence even in dx and in dy, so
// Khat(kx, ky) = sum_z w_z cos(2 pi kx dx / n) cos(2 pi ky dy / n) is real; it is formed on the
// host from a table of cos(2 pi j / n), row by row: C(|dy|, kx) = sum_dx w(dx, dy) cos(...),
// then Khat = sum_dy C(|dy|, kx) cos(...), scaled by 1 / n^2 (the inverse is unnormalised).
struct Fft64State {
    int n = 0;
    size_t batch = 0, u_dist = 0, s_dist = 0;
    cufftHandle fwd = 0, inv = 0;
    bool have_plans = false;
    double *khat = nullptr;              // [n][n/2 + 1]
    cufftDoubleComplex *spec = nullptr;  // [batch][n][n/2 + 1]
};

void fft64_release(Fft64State *f) {
    if (!f) return;
    const CufftApi &api = cufft_api();
    if (f->have_plans && api.ok) {
        api.destroy(f->fwd);
        api.destroy(f->inv);
    }
    cudaFree(f->khat);
    cudaFree(f->spec);
    delete f;
}

__global__ void fft64_multiply_kernel(cufftDoubleComplex *spec, const double *khat, size_t per, size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double k = khat[i % per];
        spec[i].x *= k;
        spec[i].y *= k;
    }
}

std::vector<double> khat64_host(const Model &m, int n) {
    const int nh1 = n / 2 + 1;
    std::vector<double> cs(n), C((size_t)(m.R + 1) * nh1, 0.0), K((size_t)n * nh1, 0.0);
    for (int j = 0; j < n; ++j) cs[j] = std::cos(2.0 * M_PI * j / n);
    for (int ady = 0; ady <= m.R; ++ady) {
        const int w = m.widths[ady];
        for (int kx = 0; kx < nh1; ++kx) {
            double c = 0.0;
            for (int dx = -w; dx <= w; ++dx) {
                const double wt = m.d.kernel == MFMC_KERNEL_CONSTANT ? 1.0 : m.wtab64[dx * dx + ady * ady];
                c += wt * cs[(size_t)(((long)kx * dx) % n + n) % n];
            }
            C[(size_t)ady * nh1 + kx] = c;
        }
    }
    const double inv_nn = 1.0 / ((double)n * n);
    for (int ky = 0; ky < n; ++ky)
        for (int kx = 0; kx < nh1; ++kx) {
            double k = 0.0;
            for (int dy = -m.R; dy <= m.R; ++dy)
                k += C[(size_t)(dy < 0 ? -dy : dy) * nh1 + kx] * cs[(size_t)(((long)ky * dy) % n + n) % n];
            K[(size_t)ky * nh1 + kx] = k * inv_nn;
        }
    return K;
}

mfmc_status fft64_disc_sums(Model &m, const double *u, size_t u_dist, double *S, size_t s_dist, size_t ns,
                            cudaStream_t st) {
    const CufftApi &api = cufft_api();
    if (!fft64_available()) return fail(MFMC_ECUDA, "cuFFT (libcufft.so) could not be loaded");
    if (ns == 0) return MFMC_OK;
    const int n = m.d.n, nh1 = n / 2 + 1;
    const size_t nh = (size_t)n * nh1;
    if (ns > (size_t)INT32_MAX || u_dist > (size_t)INT32_MAX || s_dist > (size_t)INT32_MAX)
        return fail(MFMC_EINVAL, "batch too large for the spectral disc sums");
    if (!m.fft64) m.fft64 = new Fft64State();
    Fft64State &f = *m.fft64;
    if (f.n != n) {
        const std::vector<double> K = khat64_host(m, n);
        cudaFree(f.khat);
        f.khat = nullptr;
        MFMC_CUDA(cudaMalloc((void **)&f.khat, nh * sizeof(double)));
        MFMC_CUDA(cudaMemcpy(f.khat, K.data(), nh * sizeof(double), cudaMemcpyHostToDevice));
        f.n = n;
        f.batch = 0;
    }
    if (!f.have_plans || f.batch != ns || f.u_dist != u_dist || f.s_dist != s_dist) {
        MFMC_CUDA(cudaStreamSynchronize(st));
        if (f.have_plans) {
            api.destroy(f.fwd);
            api.destroy(f.inv);
        }
        f.have_plans = false;
        cudaFree(f.spec);
        f.spec = nullptr;
        int dims[2] = {n, n}, emb_r[2] = {n, n}, emb_c[2] = {n, nh1};
        MFMC_CUFFT(api.plan_many(&f.fwd, 2, dims, emb_r, 1, (int)u_dist, emb_c, 1, (int)nh, CUFFT_D2Z, (int)ns));
        cufftResult r = api.plan_many(&f.inv, 2, dims, emb_c, 1, (int)nh, emb_r, 1, (int)s_dist, CUFFT_Z2D, (int)ns);
        if (r != CUFFT_SUCCESS) {
            api.destroy(f.fwd);
            return fail(MFMC_ECUDA, "cufftPlanMany (FP64 inverse) failed (%d)", (int)r);
        }
        f.have_plans = true;
        MFMC_CUDA(cudaMalloc((void **)&f.spec, ns * nh * sizeof(cufftDoubleComplex)));
        f.batch = ns;
        f.u_dist = u_dist;
        f.s_dist = s_dist;
    }
    MFMC_CUFFT(api.set_stream(f.fwd, st));
    MFMC_CUFFT(api.set_stream(f.inv, st));
    // cuFFT's D2Z input is non-const in its signature; an out-of-place transform does not write it
    MFMC_CUFFT(api.exec_d2z(f.fwd, const_cast<double *>(u), f.spec));
    const size_t tot = ns * nh;
    fft64_multiply_kernel<<<(unsigned)std::min<size_t>((tot + 255) / 256, 152 * 64), 256, 0, st>>>(f.spec, f.khat,
                                                                                                nh, tot);
    MFMC_LAUNCHED("fft_solver launch 4");
    MFMC_CUFFT(api.exec_z2d(f.inv, f.spec, S));
    return MFMC_OK;
}

}  // namespace mfmc
