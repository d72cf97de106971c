// Initial fields, step coefficients, the generic (any R, any radial kernel) step kernel,
// the OoI finalisation and the solve drivers for every algorithm.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "mfmc_internal.h"
#include <cudaTypedefs.h>

#include <mutex>

#include "rows_step.cuh"

namespace mfmc {

// ----------------------------------------------------------------------------- ICs
// Built in FP64 with explicitly rounded operations (no contraction) and rounded to FP32.
__device__ double ic_normal(uint64_t seed, uint32_t q) {
    const double u1 = __dsub_rn(1.0, sm64_unit(seed, 1, 2u * q));
    const double u2 = sm64_unit(seed, 1, 2u * q + 1u);
    return __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))),
                     cos(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), u2)));
}

__device__ __forceinline__ double clip1(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

// Base-lattice value of the noise ICs at node (Y, X) of the N x N lattice.
__device__ double noise_base(int N, int ic, double amp, uint64_t seed, int Y, int X) {
    const uint32_t p = (uint32_t)(Y * N + X);
    if (ic == MFMC_IC_UNIFORM) return __dmul_rn(amp, __dsub_rn(__dmul_rn(2.0, sm64_unit(seed, 1, p)), 1.0));
    const int xm = X == 0 ? N - 1 : X - 1, xp = X == N - 1 ? 0 : X + 1;
    const int ym = Y == 0 ? N - 1 : Y - 1, yp = Y == N - 1 ? 0 : Y + 1;
    double s = __dmul_rn(amp, ic_normal(seed, p));
    s = __dadd_rn(s, __dmul_rn(amp, ic_normal(seed, (uint32_t)(Y * N + xm))));
    s = __dadd_rn(s, __dmul_rn(amp, ic_normal(seed, (uint32_t)(Y * N + xp))));
    s = __dadd_rn(s, __dmul_rn(amp, ic_normal(seed, (uint32_t)(ym * N + X))));
    s = __dadd_rn(s, __dmul_rn(amp, ic_normal(seed, (uint32_t)(yp * N + X))));
    return clip1(__ddiv_rn(s, 5.0));
}

__global__ void init_fields_kernel(int n, int ic, double amp, int base_n, const uint64_t *seeds,
                                   const double *theta, size_t ns, float *u0) {
    const size_t nn = (size_t)n * n;
    const size_t total = nn * ns;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t smp = idx / nn;
        const uint32_t p = (uint32_t)(idx - smp * nn);
        const int y = p / n, x = p - (p / n) * n;
        const uint64_t seed = seeds[smp];
        double v;
        if (ic == MFMC_IC_UNIFORM || ic == MFMC_IC_SMOOTHED_GAUSS) {
            // mean of the b x b block of base-lattice values around the node
            const int B = base_n, b = base_n / n;
            double s = 0.0;
            for (int a = -(b / 2); a < b - b / 2; ++a) {
                int Y = b * y + a;
                Y = Y < 0 ? Y + B : (Y >= B ? Y - B : Y);
                for (int c = -(b / 2); c < b - b / 2; ++c) {
                    int X = b * x + c;
                    X = X < 0 ? X + B : (X >= B ? X - B : X);
                    s = __dadd_rn(s, noise_base(B, ic, amp, seed, Y, X));
                }
            }
            v = __ddiv_rn(s, __dmul_rn((double)b, (double)b));
        } else {
            // Eq. (ic): 1 - 2 sum_i mu_i exp(-36 |x - xbar_i - eta_i|^2), minimum image
            const double cx[4] = {0.25, 0.75, 0.5, 0.5};
            const double cy[4] = {0.5, 0.5, 0.25, 0.75};
            const double *th = theta + smp * 12;
            const double h = 1.0 / n;
            double s = 0.0;
            for (int k = 0; k < 4; ++k) {
                double ddx = __dsub_rn(__dmul_rn((double)x, h), __dadd_rn(cx[k], th[4 + 2 * k]));
                double ddy = __dsub_rn(__dmul_rn((double)y, h), __dadd_rn(cy[k], th[5 + 2 * k]));
                ddx = __dsub_rn(ddx, floor(__dadd_rn(ddx, 0.5)));
                ddy = __dsub_rn(ddy, floor(__dadd_rn(ddy, 0.5)));
                const double r2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                s = __dadd_rn(s, __dmul_rn(th[k], exp(__dmul_rn(-36.0, r2))));
            }
            v = clip1(__dsub_rn(1.0, __dmul_rn(2.0, s)));
        }
        u0[idx] = (float)v;
    }
}

// The smoothed Gaussian IC, tiled: one CTA builds an output tile of TO x TO nodes of one
// sample.  It evaluates amp * normal once for every base-lattice node of the tile's b x b
// blocks plus a one-node halo (the untiled kernel evaluates each normal five times, in
// FP64, which dominates the cost of building the fields), then the 5-point average of each
// base node and the b x b block means with the same operations in the same order, so the
// values are those of init_fields_kernel.
constexpr int IC_SPAN = 32;   // base nodes per tile edge (b * TO <= IC_SPAN)
constexpr int IC_NT = 256;

__global__ void __launch_bounds__(IC_NT) smoothed_ic_kernel(int n, double amp, int B, int b, int TO,
                                                            const uint64_t *seeds, size_t s0, float *u0) {
    __shared__ double zz[(IC_SPAN + 2) * (IC_SPAN + 2)];  // amp * normal, tile + halo
    __shared__ double nb[IC_SPAN * IC_SPAN];              // 5-point averages, clipped
    const int tiles_x = (n + TO - 1) / TO;
    const int ty0 = (blockIdx.x / tiles_x) * TO, tx0 = (blockIdx.x % tiles_x) * TO;
    const size_t smp = s0 + blockIdx.y;
    const uint64_t seed = seeds[smp];
    const int span = b * TO, zw = span + 2;
    const int Y0 = b * ty0 - b / 2 - 1, X0 = b * tx0 - b / 2 - 1;  // halo corner on the base lattice
    for (int i = threadIdx.x; i < zw * zw; i += IC_NT) {
        const int r = i / zw, c = i - r * zw;
        int Y = (Y0 + r) % B, X = (X0 + c) % B;
        Y = Y < 0 ? Y + B : Y;
        X = X < 0 ? X + B : X;
        zz[i] = __dmul_rn(amp, ic_normal(seed, (uint32_t)(Y * B + X)));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < span * span; i += IC_NT) {
        const int r = i / span + 1, c = i - (i / span) * span + 1;
        double v = zz[r * zw + c];
        v = __dadd_rn(v, zz[r * zw + c - 1]);
        v = __dadd_rn(v, zz[r * zw + c + 1]);
        v = __dadd_rn(v, zz[(r - 1) * zw + c]);
        v = __dadd_rn(v, zz[(r + 1) * zw + c]);
        nb[i] = clip1(__ddiv_rn(v, 5.0));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TO * TO; i += IC_NT) {
        const int oy = i / TO, ox = i - oy * TO;
        const int y = ty0 + oy, x = tx0 + ox;
        if (y >= n || x >= n) continue;
        double sacc = 0.0;
        for (int a = 0; a < b; ++a)
            for (int c = 0; c < b; ++c) sacc = __dadd_rn(sacc, nb[(oy * b + a) * span + ox * b + c]);
        u0[smp * (size_t)n * n + (size_t)y * n + x] = (float)__ddiv_rn(sacc, __dmul_rn((double)b, (double)b));
    }
}

mfmc_status launch_init_fields(const Model &m, const uint64_t *seeds_dev, const double *theta_dev,
                               size_t ns, float *u0, cudaStream_t st) {
    if (ns == 0) return MFMC_OK;
    const size_t total = (size_t)m.d.n * m.d.n * ns;
    const int block = 256;
    const size_t blocks = std::min<size_t>((total + block - 1) / block, 152 * 64);
    const int base_n = m.d.ic_base_n > 0 ? m.d.ic_base_n : m.d.n;
    const int b = base_n / m.d.n;
    if (m.d.ic == MFMC_IC_SMOOTHED_GAUSS && b <= IC_SPAN) {
        const int TO = IC_SPAN / b, tiles_x = (m.d.n + TO - 1) / TO;
        for (size_t o = 0; o < ns; o += 65535) {
            const unsigned gy = (unsigned)std::min<size_t>(65535, ns - o);
            smoothed_ic_kernel<<<dim3(tiles_x * tiles_x, gy), IC_NT, 0, st>>>(m.d.n, m.d.ic_amp, base_n, b, TO,
                                                                             seeds_dev, o, u0);
        }
        MFMC_LAUNCHED("nlch_solver launch 1 (tiled)");
        return MFMC_OK;
    }
    init_fields_kernel<<<(unsigned)blocks, block, 0, st>>>(m.d.n, (int)m.d.ic, m.d.ic_amp, base_n, seeds_dev,
                                                           theta_dev, ns, u0);
    MFMC_LAUNCHED("nlch_solver launch 1");
    return MFMC_OK;
}

// ----------------------------------------------------------------------------- coefficients
__global__ void coef_kernel(const double *eps, double eps_nominal, double ahat, double chat,
                            double tau, double beta1, double cF, size_t ns, StepCoef *out) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const double e = eps ? eps[i] : eps_nominal;
    const double e2 = e * e;
    const double cg = e2 * ahat * chat;                 // lattice c_gamma of this sample
    const double denom = 1.0 + tau * beta1 * cg;
    StepCoef c;
    c.c0 = (float)chat;
    c.c1 = (float)(tau * beta1 * e2 * ahat / denom);
    c.c2 = (float)(tau * beta1 * cF / denom);
    c.pad = 0.f;
    out[i] = c;
}

mfmc_status launch_coefficients(const Model &m, const double *eps_dev, size_t ns, StepCoef *coef,
                                cudaStream_t st) {
    if (ns == 0) return MFMC_OK;
    coef_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(eps_dev, m.d.eps, m.ahat, m.chat, m.d.tau,
                                                               m.d.beta1, m.d.c_F, ns, coef);
    MFMC_LAUNCHED("nlch_solver launch 2");
    return MFMC_OK;
}

// ----------------------------------------------------------------------------- generic step
// Any R <= 32 and any radial kernel (weights per r2 = dx^2 + dy^2).  One output per
// thread, 32 x 8 outputs per CTA; the disc is summed row by row, dy then dx ascending.
struct GenericArgs {
    const float *src;
    float *dst;
    const StepCoef *coef;
    double *partials;
    const float *wtab;  // NULL: unit weights
    int n, R, tiles_x, tiles, sample0, last;
    int collar;         // 1: points outside the lattice read uI (volume constraint), 0: periodic
    float uI;
    int r2max;          // the disc is { z : |z|^2 <= r2max } (R^2 for an integer delta / h)
};

constexpr int GEN_TX = 32, GEN_TY = 8, GEN_NT = GEN_TX * GEN_TY;

__global__ void __launch_bounds__(GEN_NT) step_generic_kernel(GenericArgs a) {
    extern __shared__ float4 smem4[];
    const int R = a.R;
    const int R4 = (R + 3) & ~3;
    const int SW = GEN_TX + 2 * R4, SW4 = SW / 4, SH = GEN_TY + 2 * R;
    float *s = reinterpret_cast<float *>(smem4);
    int *widths = reinterpret_cast<int *>(s + SH * SW);
    float *wt = reinterpret_cast<float *>(widths + (R + 1));
    __shared__ double red[GEN_NT / 32];

    const int n = a.n, tile = blockIdx.x, sample = a.sample0 + blockIdx.y;
    const int x0 = (tile % a.tiles_x) * GEN_TX, y0 = (tile / a.tiles_x) * GEN_TY;
    const size_t nn = (size_t)n * n;
    const float *__restrict__ src = a.src + (size_t)sample * nn;
    for (int idx = threadIdx.x; idx < SH * SW4; idx += GEN_NT) {
        const int r = idx / SW4, c4 = idx - r * SW4;
        const int py = y0 - R + r, px = x0 - R4 + 4 * c4;  // px, n: multiples of 4
        if (a.collar && (py < 0 || py >= n || px < 0 || px >= n)) {
            smem4[idx] = make_float4(a.uI, a.uI, a.uI, a.uI);
            continue;
        }
        const int gy = wrap_idx(py, n), gx = wrap_idx(px, n);
        smem4[idx] = __ldg(reinterpret_cast<const float4 *>(src + (size_t)gy * n + gx));
    }
    if (threadIdx.x <= R) {
        const int d = threadIdx.x;
        int w = 0;
        while ((w + 1) * (w + 1) <= a.r2max - d * d) ++w;
        widths[d] = w;
    }
    if (a.wtab)
        for (int i = threadIdx.x; i <= a.r2max; i += GEN_NT) wt[i] = a.wtab[i];
    __syncthreads();

    const int lx = threadIdx.x % GEN_TX, ly = threadIdx.x / GEN_TX;
    float S = 0.f;
    for (int dy = -R; dy <= R; ++dy) {
        const int w = widths[dy < 0 ? -dy : dy];
        const float *row = s + (ly + R + dy) * SW + lx + R4;
        if (a.wtab) {
            for (int dx = -w; dx <= w; ++dx) S = fmaf(wt[dx * dx + dy * dy], row[dx], S);
        } else {
            for (int dx = -w; dx <= w; ++dx) S += row[dx];
        }
    }
    const StepCoef cf = a.coef[sample];
    const float uc = s[(ly + R) * SW + lx + R4];
    const float sd = fmaf(-cf.c0, uc, S);
    float v = uc + fmaf(cf.c1, sd, cf.c2 * uc);
    v = fminf(1.f, fmaxf(-1.f, v));
    const int gy = y0 + ly, gx = x0 + lx;
    double part = 0.0;
    if (gy < n && gx < n) {
        a.dst[(size_t)sample * nn + (size_t)gy * n + gx] = v;
        part = v;
    }
    if (a.last) {
        const double t = block_sum_fixed<GEN_NT>(part, red);
        if (threadIdx.x == 0) a.partials[(size_t)sample * a.tiles + tile] = t;
    }
}

static size_t generic_smem(int R) {
    const int R4 = (R + 3) & ~3;
    return (size_t)(GEN_TY + 2 * R) * (GEN_TX + 2 * R4) * sizeof(float) + (R + 1) * sizeof(int) +
           (size_t)(R + 1) * (R + 1) * sizeof(float);  // weight table: r2max < (R + 1)^2
}

// ----------------------------------------------------------------------------- OoI
__global__ void finalize_ooi_kernel(const double *partials, int tiles, size_t ns, double inv_nn,
                                    double *ubar, double *ooi) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double t = 0.0;
    for (int k = 0; k < tiles; ++k) t += partials[i * tiles + k];  // tile order
    const double mean = t * inv_nn;
    if (ubar) ubar[i] = mean;
    if (ooi) ooi[i] = 0.5 * (1.0 + mean);
}

mfmc_status launch_finalize(const double *partials, int tiles, size_t ns, int n, double *ubar, double *ooi,
                            cudaStream_t st) {
    if (ns == 0) return MFMC_OK;
    finalize_ooi_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(partials, tiles, ns, 1.0 / ((double)n * n), ubar,
                                                                       ooi);
    MFMC_LAUNCHED("finalize");
    return MFMC_OK;
}

mfmc_status launch_pad(const float *u0, float *padded, int n, int G, size_t ns, cudaStream_t st) {
    const int P = n + 2 * G;
    const size_t total = ns * (size_t)P * (P / 4);
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 32);
    if (total == 0) return MFMC_OK;
    pad_fields_kernel<<<blocks, 256, 0, st>>>(u0, padded, n, G, ns, 0, 0.f);
    MFMC_LAUNCHED("pad");
    return MFMC_OK;
}

__global__ void reduce_fields_kernel(const float *u, int n, double *ubar, double *ooi) {
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

mfmc_status launch_field_ooi(const float *u, size_t ns, int n, double *ubar, double *ooi, cudaStream_t st) {
    const size_t nn = (size_t)n * n;
    for (size_t o = 0; o < ns; o += 65535) {
        const unsigned g = (unsigned)std::min<size_t>(65535, ns - o);
        reduce_fields_kernel<<<g, 256, 0, st>>>(u + o * nn, n, ubar ? ubar + o : nullptr, ooi ? ooi + o : nullptr);
    }
    MFMC_LAUNCHED("nlch_solver launch 9");
    return MFMC_OK;
}

bool algo_supported(const Model &m, int algo) {
    const bool constant = m.d.kernel == MFMC_KERNEL_CONSTANT;
    // beta2 > 0: only the active-set solver; it serves nothing else
    if (m.d.beta2 > 0.0 || algo == MFMC_ALGO_ACTIVE_SET) return m.d.beta2 > 0.0 && algo == MFMC_ALGO_ACTIVE_SET;
    if (algo == MFMC_ALGO_FFT) return m.d.bc == MFMC_BC_PERIODIC;  // any kernel, any radius
    if (algo == MFMC_ALGO_SPECTRAL) return spectral_supported(m);   // any kernel and radius, n = 1024
    if (algo == MFMC_ALGO_WEIGHTED)  // any radial kernel, integer delta / h, either boundary
        return m.integer_R && tma_launcher(m.R) != nullptr && tma_launcher(m.R)->v[kTmaWeighted].fn[3] != nullptr;
    // a non-integer delta / h: only the generic kernel, whose disc is set at run time
    if (!m.integer_R) return algo == MFMC_ALGO_PLAIN || algo == MFMC_ALGO_DIRECT;
    if (m.d.bc == MFMC_BC_COLLAR) {
        // the collar lives in the TMA kernels' ghost frame and in the generic kernel's loads
        switch (algo) {
            case MFMC_ALGO_PLAIN:
            case MFMC_ALGO_DIRECT: return true;
            case MFMC_ALGO_PREFIX_KAHAN:
            case MFMC_ALGO_PREFIX_TMA: return constant && tma_launcher(m.R) != nullptr;
            default: return false;
        }
    }
    switch (algo) {
        case MFMC_ALGO_PLAIN: return true;
        case MFMC_ALGO_DIRECT: return true;  // tile kernel (R <= 8) or the generic kernel
        case MFMC_ALGO_PREFIX: return constant && tile_launcher(m.R) != nullptr;
        case MFMC_ALGO_PREFIX_KAHAN:
        case MFMC_ALGO_PREFIX_TMA: return constant && tma_launcher(m.R) != nullptr;
        case MFMC_ALGO_ROWS: return constant && rows_supported(m, 4);
        case MFMC_ALGO_RESIDENT: {
            if (!constant || resident_launcher(m.R) == nullptr) return false;
            const int nt = resident_threads(m.d.n);
            return m.d.n % 4 == 0 && (m.d.n * m.d.n) % (4 * RES_RY) == 0 && nt >= 1 && nt <= 256 &&
                   m.d.n / 4 <= nt && resident_smem(m.d.n, m.R) <= 225 * 1024 && (m.d.n % RES_RY) == 0;
        }
        default: return false;
    }
}

static int tiles_for(const Model &m, int algo, int *tiles_x) {
    int tx = GEN_TX, ty = GEN_TY;
    const TileLauncher *L = tile_launcher(m.R);
    const bool constant = m.d.kernel == MFMC_KERNEL_CONSTANT;
    const bool tiled = constant && L && m.d.bc == MFMC_BC_PERIODIC && m.integer_R &&
                       ((algo == MFMC_ALGO_DIRECT && L->fn[0]) || algo == MFMC_ALGO_PREFIX);
    if (tiled) {
        tx = L->tx;
        ty = L->ty;
    }
    *tiles_x = (m.d.n + tx - 1) / tx;
    return *tiles_x * ((m.d.n + ty - 1) / ty);
}

static mfmc_status launch_generic(const Model &m, const GenericArgs &base, size_t s0, size_t cnt,
                                  cudaStream_t st) {
    const size_t smem = generic_smem(m.R);
    // set before every launch: the attribute is per device, and the call is cheap
    MFMC_CUDA(cudaFuncSetAttribute(step_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    for (size_t o = 0; o < cnt; o += 65535) {
        GenericArgs a = base;
        a.sample0 = (int)(s0 + o);
        const unsigned gy = (unsigned)std::min<size_t>(65535, cnt - o);
        step_generic_kernel<<<dim3(a.tiles, gy), GEN_NT, smem, st>>>(a);
    }
    MFMC_LAUNCHED("nlch_solver launch 3");
    return MFMC_OK;
}

// ----------------------------------------------------------------------------- TMA path
// Copy unpadded fields [ns][n][n] into padded scratch [ns][P][P] including the frame.
__global__ void pad_fields_kernel(const float *u, float *dst, int n, int G, size_t ns, int collar, float uI) {
    const int P = n + 2 * G, P4 = P / 4;
    const size_t total = ns * (size_t)P * P4;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t smp = idx / ((size_t)P * P4);
        const int rem = (int)(idx - smp * (size_t)P * P4);
        const int py = rem / P4, px = (rem - (rem / P4) * P4) * 4;
        float4 v;
        if (collar && (py < G || py >= G + n || px < G || px >= G + n)) {  // px, G, n: multiples of 4
            v = make_float4(uI, uI, uI, uI);
        } else {
            const int y = wrap_idx(py - G, n), x = wrap_idx(px - G, n);
            v = __ldg(reinterpret_cast<const float4 *>(u + smp * (size_t)n * n + (size_t)y * n + x));
        }
        *reinterpret_cast<float4 *>(dst + smp * (size_t)P * P + (size_t)py * P + px) = v;
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

mfmc_status encode_map(CUtensorMap *map, float *base, int P, size_t cap, int sw, int sh, int sd, int l2promo) {
    auto enc = tensor_map_encoder();
    if (!enc) return fail(MFMC_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)P, (cuuint64_t)cap};
    const cuuint64_t strides[2] = {(cuuint64_t)P * sizeof(float), (cuuint64_t)P * P * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)sw, (cuuint32_t)sh, (cuuint32_t)sd};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     l2promo >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                    : (l2promo >= 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                      : CU_TENSOR_MAP_L2_PROMOTION_NONE),
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MFMC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MFMC_OK;
}

static mfmc_status ensure_pad_scratch(Model &m, size_t ns, int box_w, int box_h, int box_d = 1, int l2promo = 256) {
    const int G = (m.R + 3) & ~3, P = m.d.n + 2 * G;
    if (!m.d_status) {
        MFMC_CUDA(cudaMalloc((void **)&m.d_status, sizeof(int)));
        MFMC_CUDA(cudaMemset(m.d_status, 0, sizeof(int)));
    }
    if (m.pad_cap < ns || !m.padA || !m.padB) {
        cudaFree(m.padA);
        cudaFree(m.padB);
        m.padA = m.padB = nullptr;
        m.pad_cap = 0;
        m.maps_valid = 0;
        const size_t bytes = ns * (size_t)P * P * sizeof(float);
        MFMC_CUDA(cudaMalloc((void **)&m.padA, bytes));
        MFMC_CUDA(cudaMalloc((void **)&m.padB, bytes));
        m.pad_cap = ns;
    }
    if (box_w == 0) return MFMC_OK;  // buffers only (the caller encodes its own maps)
    if (m.maps_valid && m.map_sw == box_w && m.map_sh == box_h && m.map_sd == box_d && m.map_l2 == l2promo)
        return MFMC_OK;
    m.maps_valid = 0;
    mfmc_status s = encode_map(&m.mapA, m.padA, P, m.pad_cap, box_w, box_h, box_d, l2promo);
    if (s == MFMC_OK) s = encode_map(&m.mapB, m.padB, P, m.pad_cap, box_w, box_h, box_d, l2promo);
    if (s != MFMC_OK) return s;
    m.map_sw = box_w;
    m.map_sh = box_h;
    m.map_sd = box_d;
    m.map_l2 = l2promo;
    m.maps_valid = 1;
    return MFMC_OK;
}

int tma_tiles(const Model &m, int variant, int *tiles_x) {
    const TmaLauncher *TL = tma_launcher(m.R);
    const TmaVariant &L = TL->v[variant];
    *tiles_x = (m.d.n + L.tx - 1) / L.tx;
    return *tiles_x * ((m.d.n + L.ty - 1) / L.ty);
}

mfmc_status tma_alloc_buffers(const Model &m, int variant, size_t ns, TmaBuffers *b, cudaStream_t alloc_st) {
    const TmaLauncher *TL = tma_launcher(m.R);
    if (!TL) return fail(MFMC_EINVAL, "no TMA kernel for R = %d", m.R);
    const TmaVariant &L = TL->v[variant];
    const int G = (m.R + 3) & ~3, P = m.d.n + 2 * G;
    int tiles_x = 0;
    const int tiles = tma_tiles(m, variant, &tiles_x);
    const size_t bytes = ns * (size_t)P * P * sizeof(float);
    // stream-ordered allocations: no device-wide synchronisation
    MFMC_CUDA(cudaMallocAsync((void **)&b->padA, bytes, alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->padB, bytes, alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->partials, ns * (size_t)tiles * sizeof(double), alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->status, sizeof(int), alloc_st));
    MFMC_CUDA(cudaMemsetAsync(b->status, 0, sizeof(int), alloc_st));
    b->cap = ns;
    mfmc_status s = encode_map(&b->mapA, b->padA, P, ns, L.sw, L.sh);
    if (s == MFMC_OK) s = encode_map(&b->mapB, b->padB, P, ns, L.sw, L.sh);
    return s;
}

void tma_free_buffers(TmaBuffers *b, cudaStream_t st) {
    if (b->padA) cudaFreeAsync(b->padA, st);
    if (b->padB) cudaFreeAsync(b->padB, st);
    if (b->partials) cudaFreeAsync(b->partials, st);
    if (b->status) cudaFreeAsync(b->status, st);
    b->padA = b->padB = nullptr;
    b->partials = nullptr;
    b->status = nullptr;
}

mfmc_status run_solve_tma_core(const Model &m, int kahan, int variant, const StepCoef *coef, const float *u0,
                               size_t ns, int nsteps, const int *steps_ps, float *uT, double *ubar, double *ooi,
                               const TmaBuffers &b, cudaStream_t st) {
    const TmaLauncher *TL = tma_launcher(m.R);
    if (!TL) return fail(MFMC_EINVAL, "no TMA kernel for R = %d", m.R);
    if (kahan) variant = 0;
    const int fsel = variant == kTmaWeighted ? 3 : (kahan ? 2 : 1);
    if (variant < 0 || variant > kTmaWeighted || !TL->v[variant].fn[fsel])
        return fail(MFMC_EINVAL, "TMA variant %d unavailable", variant);
    if (fsel == 3 && !m.d_wsq) return fail(MFMC_EINVAL, "the weighted form needs the model's weight table");
    const TmaVariant *L = &TL->v[variant];
    const int n = m.d.n, G = (m.R + 3) & ~3, P = n + 2 * G;
    int tiles_x = 0;
    const int tiles = tma_tiles(m, variant, &tiles_x);
    {
        const size_t total = ns * (size_t)P * (P / 4);
        const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 32);
        const int collar = m.d.bc == MFMC_BC_COLLAR;
        pad_fields_kernel<<<blocks, 256, 0, st>>>(u0, b.padB, n, G, ns, collar, (float)m.d.bc_value);
        // with a collar the steps store interior points only, so the frame of the other
        // buffer must hold the collar too (its interior is overwritten by step 1)
        if (collar) pad_fields_kernel<<<blocks, 256, 0, st>>>(u0, b.padA, n, G, ns, collar, (float)m.d.bc_value);
        MFMC_LAUNCHED("nlch_solver launch 4");
    }
    int dev = 0, sms = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long total = (long long)ns * tiles;
    if (total > (1ll << 30)) return fail(MFMC_EINVAL, "too many tiles in one solve");
    const int grid = (int)std::min<long long>(total, (long long)sms * L->blocks_per_sm());
    const CUtensorMap *src = &b.mapB;
    float *dstbuf = b.padA;
    for (int k = 1; k <= nsteps; ++k) {
        const bool last = k == nsteps;
        TmaArgs a;
        a.dst = (last && !steps_ps) ? nullptr : dstbuf;
        a.dst_plain = (last && !steps_ps) ? uT : nullptr;
        a.coef = coef;
        a.partials = b.partials;
        a.status = b.status;
        a.steps_ps = steps_ps;
        a.step = k;
        a.n = n;
        a.P = P;
        a.tiles_x = tiles_x;
        a.tiles = tiles;
        a.total = (int)total;
        a.last = (last && !steps_ps) ? 1 : 0;
        a.periodic = m.d.bc == MFMC_BC_PERIODIC;
        a.wsq = fsel == 3 ? m.d_wsq : nullptr;
        mfmc_status s = L->fn[fsel](*src, a, grid, st);
        if (s != MFMC_OK) return s;
        src = (dstbuf == b.padA) ? &b.mapA : &b.mapB;
        dstbuf = (dstbuf == b.padA) ? b.padB : b.padA;
    }
    finalize_ooi_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(b.partials, tiles, ns,
                                                                       1.0 / ((double)n * n), ubar, ooi);
    MFMC_LAUNCHED("nlch_solver launch 5");
    return MFMC_OK;
}

mfmc_status run_solve_tma(Model &m, int kahan, int variant, const StepCoef *coef, const float *u0, size_t ns,
                          int nsteps, float *uT, double *ubar, double *ooi, cudaStream_t st) {
    const TmaLauncher *TL = tma_launcher(m.R);
    if (!TL) return fail(MFMC_EINVAL, "no TMA kernel for R = %d", m.R);
    if (kahan) variant = 0;
    if (variant == kTmaWeighted) {
        if (!algo_supported(m, MFMC_ALGO_WEIGHTED)) return fail(MFMC_EINVAL, "no weighted TMA kernel for R = %d", m.R);
        if (!m.d_wsq) {
            MFMC_CUDA(cudaMalloc((void **)&m.d_wsq, m.wsq.size() * sizeof(float)));
            MFMC_CUDA(cudaMemcpy(m.d_wsq, m.wsq.data(), m.wsq.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    } else if (variant < 0 || variant >= kTmaVariants) {
        return fail(MFMC_EINVAL, "TMA variant %d unavailable", variant);
    }
    int tiles_x = 0;
    const int tiles = tma_tiles(m, variant, &tiles_x);
    mfmc_status s = ensure_pad_scratch(m, ns, TL->v[variant].sw, TL->v[variant].sh);
    if (s == MFMC_OK) s = grow_buffer(&m.partials, &m.partials_cap, ns * (size_t)tiles);
    if (s != MFMC_OK) return s;
    TmaBuffers b;
    b.padA = m.padA;
    b.padB = m.padB;
    b.mapA = m.mapA;
    b.mapB = m.mapB;
    b.cap = m.pad_cap;
    b.partials = m.partials;
    b.status = m.d_status;
    return run_solve_tma_core(m, kahan, variant, coef, u0, ns, nsteps, nullptr, uT, ubar, ooi, b, st);
}

// ----------------------------------------------------------------------------- row streaming
// Partials of the row-streaming kernel: one FP64 row sum per (sample, strip, row).
static int rows_partials_per_sample(const Model &m) { return (m.d.n / 128) * m.d.n; }

__global__ void rows_ooi_kernel(const float *plain, const float *fieldA, const float *fieldB, const int *steps_ps,
                                int nsteps, int n, int strips, size_t ns, double *partials) {
    const int lane = threadIdx.x & 31;
    const long long total = (long long)ns * strips * n;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total; r += warps) {
        const long long col = r / n;
        const int y = (int)(r - col * n);
        const int sample = (int)(col / strips), strip = (int)(col - (long long)sample * strips);
        const int ks = steps_ps ? steps_ps[sample] : nsteps;
        const float *f = plain ? plain : ((ks & 1) ? fieldA : fieldB);
        const float4 v = *reinterpret_cast<const float4 *>(f + (size_t)sample * n * n + (size_t)y * n + 128 * strip +
                                                           4 * lane);
        double rs = ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
        for (int off = 16; off > 0; off >>= 1) rs += __shfl_down_sync(0xffffffffu, rs, off);
        if (lane == 0) partials[r] = rs;
    }
}

// Geometry of the row-streaming kernel: 16 warps per CTA at most, n / 128 warps per sample, a
// row of n floats read through a 4-D view (k pieces of n / k <= 256 floats, n / k a multiple of
// 4 so each piece is a whole number of 16-byte units).
static bool rows_geom(const Model &m, RowsGeom *g) {
    const int n = m.d.n;
    if (n % 128 != 0 || n > 2048) return false;
    g->strips = n / 128;
    g->gs = 16 / g->strips;
    g->warps = g->gs * g->strips;
    g->k = 0;
    for (int k = 1; k <= 64; ++k)
        if (n % k == 0 && n / k <= 256 && (n / k) % 4 == 0) {
            g->k = k;
            break;
        }
    if (g->k == 0) return false;
    const RowsLauncher *L = rows_launcher(m.R);
    if (!L) return false;
    g->stage_floats = g->gs * L->ch * n;
    g->smem = (size_t)L->nstg * g->stage_floats * sizeof(float) + 128;
    return g->smem <= 227 * 1024;
}

// Tensor map of the fields [cap][n][n] as (n / k, k, cap, n): a box of (n / k, k, gs, rows) is
// `rows` whole rows of gs samples, stored in shared memory as [row][sample][n].
static mfmc_status encode_rows_map(CUtensorMap *map, float *base, const Model &m, const RowsGeom &g, size_t cap,
                                   int rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return fail(MFMC_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const int n = m.d.n, w = n / g.k;
    const cuuint64_t dims[4] = {(cuuint64_t)w, (cuuint64_t)g.k, (cuuint64_t)cap, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)w * sizeof(float), (cuuint64_t)n * n * sizeof(float),
                                   (cuuint64_t)n * sizeof(float)};
    const cuuint32_t box[4] = {(cuuint32_t)w, (cuuint32_t)g.k, (cuuint32_t)g.gs, (cuuint32_t)rows};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MFMC_ECUDA, "cuTensorMapEncodeTiled (rows) failed (%d)", (int)r);
    return MFMC_OK;
}

static mfmc_status encode_rows_maps(TmaBuffers *b, const Model &m, const RowsGeom &g, int ch) {
    mfmc_status s = encode_rows_map(&b->mapA, b->padA, m, g, b->cap, ch);
    if (s == MFMC_OK) s = encode_rows_map(&b->mapA1, b->padA, m, g, b->cap, 1);
    if (s == MFMC_OK) s = encode_rows_map(&b->mapB, b->padB, m, g, b->cap, ch);
    if (s == MFMC_OK) s = encode_rows_map(&b->mapB1, b->padB, m, g, b->cap, 1);
    return s;
}

mfmc_status rows_alloc_buffers(const Model &m, int bh, size_t ns, TmaBuffers *b, cudaStream_t alloc_st) {
    const RowsLauncher *L = rows_launcher(m.R);
    RowsGeom g;
    if (!L || !rows_geom(m, &g)) return fail(MFMC_EINVAL, "no row-streaming kernel for n = %d, R = %d", m.d.n, m.R);
    if (bh != 0 && bh < 8) return fail(MFMC_EINVAL, "band height %d < 8", bh);
    const size_t bytes = ns * (size_t)m.d.n * m.d.n * sizeof(float);
    MFMC_CUDA(cudaMallocAsync((void **)&b->padA, bytes, alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->padB, bytes, alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->partials, ns * (size_t)rows_partials_per_sample(m) * sizeof(double),
                              alloc_st));
    MFMC_CUDA(cudaMallocAsync((void **)&b->status, sizeof(int), alloc_st));
    MFMC_CUDA(cudaMemsetAsync(b->status, 0, sizeof(int), alloc_st));
    b->cap = ns;
    return encode_rows_maps(b, m, g, L->ch);
}

// The row-streaming kernel: constant kernel, periodic lattice, integer R <= 8, 128-column strips
// (n % 128 == 0, n <= 2048), four columns per thread.
bool rows_supported(const Model &m, int rx) {
    RowsGeom g;
    return m.d.kernel == MFMC_KERNEL_CONSTANT && m.d.bc == MFMC_BC_PERIODIC && m.integer_R && rx == 4 &&
           rows_launcher(m.R) != nullptr && rows_geom(m, &g);
}

mfmc_status run_solve_rows_core(const Model &m, int bh, int rx, const StepCoef *coef, const float *u0, size_t ns,
                                int nsteps, const int *steps_ps, float *uT, double *ubar, double *ooi,
                                const TmaBuffers &b, cudaStream_t st) {
    if (!rows_supported(m, rx)) return fail(MFMC_EINVAL, "row-streaming kernel unsupported (n = %d, R = %d, %d columns)", m.d.n, m.R, rx);
    const RowsLauncher *L = rows_launcher(m.R);
    RowsGeom g;
    rows_geom(m, &g);
    if (bh != 0 && bh < 8) return fail(MFMC_EINVAL, "band height %d < 8", bh);
    const int n = m.d.n;
    // B holds the fields after an even number of steps: step 0 is the initial field
    MFMC_CUDA(cudaMemcpyAsync(b.padB, u0, ns * (size_t)n * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    int dev = 0, sms = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long rows = (long long)((ns + g.gs - 1) / g.gs) * n;  // (sample group, row) order
    if (rows == 0) return MFMC_OK;
    if (rows / n * (n + 2LL * m.R) >= (1LL << 31) || (bh > 0 && rows + bh >= (1LL << 31)))
        return fail(MFMC_EINVAL, "batch of %zu samples too large for the row-streaming kernel", ns);
    // one range per CTA (at least 4R + 8 rows each, so the halo rows stay a minor share), or
    // bands taken in turn by the resident CTAs
    const int threads = 32 * g.warps;
    const long long ctas = bh > 0 ? (rows + bh - 1) / bh : rows / (4 * m.R + 8) + 1;
    const int grid =
        (int)std::max<long long>(1, std::min<long long>((long long)sms * L->blocks_per_sm(threads, g.smem), ctas));
    bool fromB = true;
    float *dstbuf = b.padA;
    for (int k = 1; k <= nsteps; ++k) {
        const bool last = k == nsteps;
        RowsArgs a;
        // the last step stores to the caller's field when asked, else to the scratch field, from
        // which rows_ooi_kernel reduces the OoI
        a.t.dst = (last && !steps_ps && uT) ? uT : dstbuf;
        a.t.dst_plain = nullptr;
        a.t.coef = coef;
        a.t.partials = b.partials;
        a.t.status = b.status;
        a.t.steps_ps = steps_ps;
        a.t.step = k;
        a.t.n = n;
        a.t.P = n;
        a.t.tiles_x = g.strips;
        a.t.tiles = g.strips * n;
        a.t.total = 0;
        a.t.last = 0;
        a.t.periodic = 1;
        a.t.wsq = nullptr;
        a.ns = (int)ns;
        a.gs = g.gs;
        a.strips = g.strips;
        a.rows = rows;
        a.band = bh;
        a.halo = 2 * m.R;
        a.stage_floats = g.stage_floats;
        a.pitch = g.gs * n;
        a.ng = 1;  // one lockstep group per CTA (measured faster than two or four)
        // steps after the first follow a step: programmatic dependents of it
        mfmc_status s = L->fn(fromB ? b.mapB : b.mapA, fromB ? b.mapB1 : b.mapA1, a, grid, threads, g.smem, k > 1, st);
        if (s != MFMC_OK) return s;
        fromB = !fromB;
        dstbuf = (dstbuf == b.padA) ? b.padB : b.padA;
    }
    {
        const long long warps = std::min<long long>((long long)ns * g.strips * n, (long long)sms * 64);
        const unsigned blocks = (unsigned)std::max<long long>(1, (warps + 7) / 8);
        rows_ooi_kernel<<<blocks, 256, 0, st>>>((uT && !steps_ps) ? uT : nullptr, b.padA, b.padB, steps_ps, nsteps,
                                                n, g.strips, ns, b.partials);
        MFMC_LAUNCHED("nlch_solver launch 7a");
    }
    finalize_ooi_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(b.partials, g.strips * n, ns,
                                                                       1.0 / ((double)n * n), ubar, ooi);
    MFMC_LAUNCHED("nlch_solver launch 7");
    return MFMC_OK;
}

mfmc_status run_solve_rows(Model &m, int bh, int rx, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                           float *uT, double *ubar, double *ooi, cudaStream_t st) {
    const RowsLauncher *L = rows_launcher(m.R);
    RowsGeom g;
    if (!L || !rows_geom(m, &g)) return fail(MFMC_EINVAL, "no row-streaming kernel for n = %d, R = %d", m.d.n, m.R);
    if (bh != 0 && bh < 8) return fail(MFMC_EINVAL, "band height %d < 8", bh);
    // the model's scratch buffers (sized for ghost-framed fields; used here as plain fields),
    // with tensor maps of the row view
    mfmc_status s = ensure_pad_scratch(m, ns, 0, 0);
    if (s == MFMC_OK) s = grow_buffer(&m.partials, &m.partials_cap, ns * (size_t)rows_partials_per_sample(m));
    if (s != MFMC_OK) return s;
    TmaBuffers b;
    b.padA = m.padA;
    b.padB = m.padB;
    b.cap = m.pad_cap;
    b.partials = m.partials;
    b.status = m.d_status;
    s = encode_rows_maps(&b, m, g, L->ch);
    if (s != MFMC_OK) return s;
    return run_solve_rows_core(m, bh, rx, coef, u0, ns, nsteps, nullptr, uT, ubar, ooi, b, st);
}

mfmc_status run_resident_steps(const Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                               const int *steps_ps, float *uT, double *ubar, double *ooi, cudaStream_t st) {
    ResidentArgs a;
    a.u0 = u0;
    a.uT = uT;
    a.coef = coef;
    a.ubar = ubar;
    a.ooi = ooi;
    a.steps_ps = steps_ps;
    a.n = m.d.n;
    a.ns = (int)ns;
    a.nsteps = nsteps;
    ResidentFn f = resident_launcher(m.R);
    if (!f) return fail(MFMC_EINVAL, "no resident kernel for R = %d", m.R);
    return f(a, st);
}

mfmc_status run_solve(Model &m, int algo, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                      float *uT, double *ubar, double *ooi, cudaStream_t st) {
    if (ns == 0) return MFMC_OK;
    const int n = m.d.n;
    const size_t nn = (size_t)n * n;
    if (!algo_supported(m, algo)) return fail(MFMC_EINVAL, "algorithm %d does not support this model", algo);
    if (nsteps == 0) {
        if (uT) MFMC_CUDA(cudaMemcpyAsync(uT, u0, nn * ns * sizeof(float), cudaMemcpyDeviceToDevice, st));
        for (size_t o = 0; o < ns; o += 65535) {
            const unsigned g = (unsigned)std::min<size_t>(65535, ns - o);
            reduce_fields_kernel<<<g, 256, 0, st>>>(u0 + o * nn, n, ubar ? ubar + o : nullptr,
                                                    ooi ? ooi + o : nullptr);
        }
        MFMC_LAUNCHED("nlch_solver launch 8");
        return MFMC_OK;
    }
    if (algo == MFMC_ALGO_FFT) return run_solve_fft(m, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_SPECTRAL) return run_solve_spectral(m, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_WEIGHTED) return run_solve_tma(m, 0, kTmaWeighted, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_PREFIX_TMA)
        return run_solve_tma(m, 0, m.tma_variant, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_PREFIX_KAHAN) return run_solve_tma(m, 1, 0, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_ROWS) return run_solve_rows(m, m.rows_bh, 4, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (algo == MFMC_ALGO_RESIDENT) return run_resident_steps(m, coef, u0, ns, nsteps, nullptr, uT, ubar, ooi, st);
    int tiles_x = 0;
    const int tiles = tiles_for(m, algo, &tiles_x);
    mfmc_status s = ensure_scratch(m, ns, (size_t)tiles);
    if (s != MFMC_OK) return s;

    const bool constant = m.d.kernel == MFMC_KERNEL_CONSTANT;
    const TileLauncher *L = tile_launcher(m.R);
    const int ai = algo == MFMC_ALGO_DIRECT ? 0 : 1;
    const bool tiled =
        algo != MFMC_ALGO_PLAIN && constant && L && L->fn[ai] && m.d.bc == MFMC_BC_PERIODIC && m.integer_R;

    if (algo == MFMC_ALGO_PLAIN) {
        // reference form: one sample per launch, one launch per step
        for (size_t smp = 0; smp < ns; ++smp) {
            const float *src = u0;
            for (int k = 1; k <= nsteps; ++k) {
                float *dst = (k == nsteps && uT) ? uT : ((k & 1) ? m.bufA : m.bufB);
                GenericArgs g;
                g.src = src;
                g.dst = dst;
                g.coef = coef;
                g.partials = m.partials;
                g.wtab = constant ? nullptr : m.d_wtab;
                g.n = n;
                g.R = m.R;
                g.tiles_x = tiles_x;
                g.tiles = tiles;
                g.sample0 = 0;
                g.last = k == nsteps;
                g.collar = m.d.bc == MFMC_BC_COLLAR;
                g.uI = (float)m.d.bc_value;
                g.r2max = m.r2max;
                s = launch_generic(m, g, smp, 1, st);
                if (s != MFMC_OK) return s;
                src = dst;
            }
        }
    } else {
        const float *src = u0;
        for (int k = 1; k <= nsteps; ++k) {
            float *dst = (k == nsteps && uT) ? uT : ((k & 1) ? m.bufA : m.bufB);
            if (tiled) {
                TileArgs t;
                t.src = src;
                t.dst = dst;
                t.coef = coef;
                t.partials = m.partials;
                t.n = n;
                t.tiles_x = tiles_x;
                t.tiles = tiles;
                t.sample0 = 0;
                t.last = k == nsteps;
                s = L->fn[ai](t, ns, st);
            } else {
                GenericArgs g;
                g.src = src;
                g.dst = dst;
                g.coef = coef;
                g.partials = m.partials;
                g.wtab = constant ? nullptr : m.d_wtab;
                g.n = n;
                g.R = m.R;
                g.tiles_x = tiles_x;
                g.tiles = tiles;
                g.sample0 = 0;
                g.last = k == nsteps;
                g.collar = m.d.bc == MFMC_BC_COLLAR;
                g.uI = (float)m.d.bc_value;
                g.r2max = m.r2max;
                s = launch_generic(m, g, 0, ns, st);
            }
            if (s != MFMC_OK) return s;
            src = dst;
        }
    }
    finalize_ooi_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(m.partials, tiles, ns, 1.0 / (double)nn,
                                                                       ubar, ooi);
    MFMC_LAUNCHED("nlch_solver launch 9");
    return MFMC_OK;
}

}  // namespace mfmc
