// mfmc_solve_fields_noalloc: the solve of mfmc_solve_fields with its scratch (two field
// buffers, step coefficients, per-tile OoI partials) in one fixed device array of this
// file instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory when they solve: a process whose framework
// reserves all device memory up front through its own allocator, or a latency-critical
// loop that must not pay for (or risk the failure of) a cudaMalloc, which can synchronise
// the device.  This entry point allocates nothing: the array below is part of the
// library's device image, so every GPU that loads the library holds it until exit.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "mfmc_internal.h"
#include "step_kernels.cuh"

namespace mfmc {

// Layout: [coefficients: kNaMaxSamples x 16 B][partials: kNaMaxPartials x 8 B][field A][field B]
constexpr size_t kNaBytes = 32ull << 20;
constexpr size_t kNaMaxSamples = 4096;
constexpr size_t kNaMaxPartials = 65536;
constexpr size_t kNaCoefBytes = kNaMaxSamples * sizeof(StepCoef);
constexpr size_t kNaPartialBytes = kNaMaxPartials * sizeof(double);
constexpr size_t kNaFieldBytes = (kNaBytes - kNaCoefBytes - kNaPartialBytes) / 2 / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the array on each device, looked up once per device.
constexpr int kNaMaxDevices = 64;
static unsigned char *g_na_ptr[kNaMaxDevices];
static std::mutex g_na_mu;

static mfmc_status noalloc_base(unsigned char **out) {
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(MFMC_EINVAL, "device %d beyond the supported range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return MFMC_OK;
}

__global__ void na_finalize_kernel(const double *partials, int tiles, size_t ns, double inv_nn, double *ubar,
                                   double *ooi) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double t = 0.0;
    for (int k = 0; k < tiles; ++k) t += partials[i * tiles + k];
    const double mean = t * inv_nn;
    if (ubar) ubar[i] = mean;
    if (ooi) ooi[i] = 0.5 * (1.0 + mean);
}

__global__ void na_reduce_kernel(const float *u, int n, double *ubar, double *ooi) {
    __shared__ double red[256];
    const size_t nn = (size_t)n * n;
    const float *f = u + blockIdx.x * nn;
    double t = 0.0;
    for (size_t i = threadIdx.x; i < nn; i += 256) t += f[i];
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

}  // namespace mfmc

using namespace mfmc;

extern "C" mfmc_status mfmc_solve_fields_noalloc(const mfmc_model *cm, const double *eps, const float *u0,
                                                 size_t ns, float *uT, double *ubar, double *ooi, void *stream) {
    if (!cm) return fail(MFMC_EINVAL, "NULL model");
    if (ns == 0) return MFMC_OK;
    if (!u0) return fail(MFMC_EINVAL, "NULL u0");
    if (uT && uT == u0) return fail(MFMC_EINVAL, "uT must not alias u0");
    const Model &m = *cm;
    const TileLauncher *L = tile_launcher(m.R);
    if (m.d.kernel != MFMC_KERNEL_CONSTANT || m.d.bc != MFMC_BC_PERIODIC || !m.integer_R || m.d.beta2 > 0.0 || !L)
        return fail(MFMC_EINVAL, "the allocation-free solve supports the periodic constant kernel with R in "
                                 "{1,2,3,4,5,6,8,11,12,16,22,24,32}");
    const int n = m.d.n;
    const size_t field = (size_t)n * n * sizeof(float);
    const int tiles_x = (n + L->tx - 1) / L->tx;
    const int tiles = tiles_x * ((n + L->ty - 1) / L->ty);
    if (ns > kNaMaxSamples || ns * field > kNaFieldBytes || ns * (size_t)tiles > kNaMaxPartials)
        return fail(MFMC_EINVAL,
                    "batch too large for the fixed scratch: ns = %zu fields of %zu bytes need %zu bytes per "
                    "buffer (limit %zu bytes, at most %zu samples and %zu tile partials)",
                    ns, field, ns * field, kNaFieldBytes, kNaMaxSamples, kNaMaxPartials);
    unsigned char *base = nullptr;
    mfmc_status s = noalloc_base(&base);
    if (s != MFMC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    StepCoef *coef = reinterpret_cast<StepCoef *>(base);
    double *partials = reinterpret_cast<double *>(base + kNaCoefBytes);
    float *fa = reinterpret_cast<float *>(base + kNaCoefBytes + kNaPartialBytes);
    float *fb = reinterpret_cast<float *>(base + kNaCoefBytes + kNaPartialBytes + kNaFieldBytes);

    s = launch_coefficients(m, eps, ns, coef, st);
    if (s != MFMC_OK) return s;
    const int nsteps = m.d.nsteps;
    if (nsteps == 0) {
        if (uT) MFMC_CUDA(cudaMemcpyAsync(uT, u0, ns * field, cudaMemcpyDeviceToDevice, st));
        for (size_t o = 0; o < ns; o += 65535) {
            const unsigned g = (unsigned)std::min<size_t>(65535, ns - o);
            na_reduce_kernel<<<g, 256, 0, st>>>(u0 + o * (size_t)n * n, n, ubar ? ubar + o : nullptr,
                                               ooi ? ooi + o : nullptr);
        }
        MFMC_LAUNCHED("noalloc launch 1");
        return MFMC_OK;
    }
    // every tile partial is rewritten at the last step, so nothing needs clearing
    const float *src = u0;
    for (int k = 1; k <= nsteps; ++k) {
        float *dst = (k == nsteps && uT) ? uT : ((k & 1) ? fa : fb);
        TileArgs t;
        t.src = src;
        t.dst = dst;
        t.coef = coef;
        t.partials = partials;
        t.n = n;
        t.tiles_x = tiles_x;
        t.tiles = tiles;
        t.sample0 = 0;
        t.last = k == nsteps;
        s = L->fn[1](t, ns, st);
        if (s != MFMC_OK) return s;
        src = dst;
    }
    na_finalize_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(partials, tiles, ns, 1.0 / ((double)n * n), ubar,
                                                                       ooi);
    MFMC_LAUNCHED("noalloc launch 2");
    return MFMC_OK;
}
