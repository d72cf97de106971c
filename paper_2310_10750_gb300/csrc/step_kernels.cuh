// Fused step kernels of the nonlocal Cahn-Hilliard scheme (beta2 = 0):
//   disc sum over the horizon (Eq. nonl_operator, lattice quadrature)
//   -> implicit-convex / explicit-concave update and projection onto [-1, 1]
//      (Eq. nonl_CH_nm, Eq. potential_obstacle)
//   -> at the last step, the per-tile partial of the output of interest (Eq. ooi).
//
// Data layout: FP32 fields, row-major [sample][y][x], n % 4 == 0, periodic.  Every
// kernel stages a tile plus an R-row / R4-column halo (R4 = R rounded up to a multiple
// of 4) in shared memory with 16-byte coalesced loads, wrapping indices at the torus
// edges, then each thread produces a 4 x RY register block of outputs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mfmc_internal.h"

namespace mfmc {

// Index on the torus.  Tiles may be wider or taller than the lattice (n = 64 with a
// 128-row tile), so the correction loops until v is in [0, n); usually it runs 0 or 1 times.
__device__ __forceinline__ int wrap_idx(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// Half widths w(|dy|) = floor(sqrt(R^2 - dy^2)) of the disc rows.
template <int R>
struct DiscRows {
    int w[R + 1];
    constexpr DiscRows() : w() {
        for (int d = 0; d <= R; ++d) {
            int s = 0;
            while ((s + 1) * (s + 1) <= R * R - d * d) ++s;
            w[d] = s;
        }
    }
};

// Classes of disc rows by half-width.  The half-widths do not increase with |dy|, so rows
// of equal half-width are consecutive; a class's row segment sum is the same for every
// output row that a staged row serves through that class.
template <int R>
struct DiscClasses {
    int count;       // number of distinct half-widths
    int width[R + 1];  // half-width of class c (decreasing in c)
    int of[R + 1];     // class of |dy|
    constexpr DiscClasses() : count(0), width(), of() {
        const DiscRows<R> d{};
        for (int a = 0; a <= R; ++a) {
            if (a == 0 || d.w[a] != d.w[a - 1]) width[count++] = d.w[a];
            of[a] = count - 1;
        }
    }
};

struct TileArgs {
    const float *src;
    float *dst;
    const StepCoef *coef;
    double *partials;  // [ns][tiles] at the last step, else unused
    int n;
    int tiles_x;
    int tiles;
    int sample0;
    int last;
};

// Block-wide FP64 sum with a fixed reduction order (deterministic).
template <int NT>
__device__ __forceinline__ double block_sum_fixed(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (NT + 31) / 32; ++i) t += red[i];
    return t;  // valid in thread 0
}

// ALGO: 0 direct disc sum, 1 in-register row prefix sums, 2 prefix + Kahan-compensated
// accumulation of the row segments.
template <int R, int RY, int TXT, int TYT, int ALGO>
__global__ void __launch_bounds__(TXT *TYT) step_tile_kernel(TileArgs a) {
    constexpr int RX = 4;
    constexpr int R4 = (R + 3) & ~3;
    constexpr int TX = RX * TXT;
    constexpr int TY = RY * TYT;
    constexpr int SW = TX + 2 * R4;
    constexpr int SW4 = SW / 4;
    constexpr int SH = TY + 2 * R;
    constexpr int NT = TXT * TYT;
    constexpr int WIN = RX + 2 * R4;  // floats a thread reads per row
    constexpr DiscRows<R> disc{};

    extern __shared__ float4 smem4[];
    float *s = reinterpret_cast<float *>(smem4);
    __shared__ double red[(NT + 31) / 32];

    const int n = a.n;
    const int tile = blockIdx.x;
    const int sample = a.sample0 + blockIdx.y;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = (tile / a.tiles_x) * TY;
    const size_t nn = (size_t)n * n;
    const float *__restrict__ src = a.src + (size_t)sample * nn;
    float *__restrict__ dst = a.dst + (size_t)sample * nn;

    // stage tile + halo, 16 B per load, indices wrapped on the torus
    for (int idx = threadIdx.x; idx < SH * SW4; idx += NT) {
        const int r = idx / SW4;
        const int c4 = idx - r * SW4;
        const int gy = wrap_idx(y0 - R + r, n);
        const int gx = wrap_idx(x0 - R4 + 4 * c4, n);
        smem4[idx] = __ldg(reinterpret_cast<const float4 *>(src + (size_t)gy * n + gx));
    }
    __syncthreads();

    const int tx = threadIdx.x % TXT;
    const int ty = threadIdx.x / TXT;
    const int ox = tx * RX;
    const int oy = ty * RY;

    float acc[RY][RX];
    float cmp[ALGO == 2 ? RY : 1][RX];
#pragma unroll
    for (int j = 0; j < RY; ++j)
#pragma unroll
        for (int i = 0; i < RX; ++i) {
            acc[j][i] = 0.f;
            cmp[ALGO == 2 ? j : 0][i] = 0.f;
        }

#pragma unroll
    for (int r = 0; r < RY + 2 * R; ++r) {
        const float4 *rowp = reinterpret_cast<const float4 *>(s + (oy + r) * SW + ox);
        float v[WIN];
#pragma unroll
        for (int q = 0; q < WIN / 4; ++q) {
            const float4 t = rowp[q];
            v[4 * q + 0] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
        if (ALGO == 0) {
#pragma unroll
            for (int j = 0; j < RY; ++j) {
                const int dy = r - R - j;
                if (dy >= -R && dy <= R) {
                    const int w = disc.w[dy < 0 ? -dy : dy];
#pragma unroll
                    for (int i = 0; i < RX; ++i) {
                        float h = 0.f;
#pragma unroll
                        for (int dx = -R; dx <= R; ++dx)
                            if (dx >= -w && dx <= w) h += v[R4 + i + dx];
                        acc[j][i] += h;
                    }
                }
            }
        } else {
            // window index k covers columns R4 - R + k, k = 0 .. RX + 2R - 1
            float p[RX + 2 * R + 1];
            p[0] = 0.f;
#pragma unroll
            for (int k = 0; k < RX + 2 * R; ++k) p[k + 1] = p[k] + v[R4 - R + k];
#pragma unroll
            for (int j = 0; j < RY; ++j) {
                const int dy = r - R - j;
                if (dy >= -R && dy <= R) {
                    const int w = disc.w[dy < 0 ? -dy : dy];
#pragma unroll
                    for (int i = 0; i < RX; ++i) {
                        const float h = p[i + R + w + 1] - p[i + R - w];
                        if (ALGO == 1) {
                            acc[j][i] += h;
                        } else {
                            const float y = h - cmp[ALGO == 2 ? j : 0][i];
                            const float t = acc[j][i] + y;
                            cmp[ALGO == 2 ? j : 0][i] = (t - acc[j][i]) - y;
                            acc[j][i] = t;
                        }
                    }
                }
            }
        }
    }

    const StepCoef cf = a.coef[sample];
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < RY; ++j) {
        const float4 c4v = *reinterpret_cast<const float4 *>(s + (oy + j + R) * SW + ox + R4);
        const float uc[4] = {c4v.x, c4v.y, c4v.z, c4v.w};
        float o[4];
#pragma unroll
        for (int i = 0; i < RX; ++i) {
            const float sd = fmaf(-cf.c0, uc[i], acc[j][i]);
            const float v = uc[i] + fmaf(cf.c1, sd, cf.c2 * uc[i]);
            o[i] = fminf(1.f, fmaxf(-1.f, v));
        }
        const int gy = y0 + oy + j;
        const int gx = x0 + ox;
        if (gy < n && gx < n) {
            *reinterpret_cast<float4 *>(dst + (size_t)gy * n + gx) = make_float4(o[0], o[1], o[2], o[3]);
            if (a.last) part += ((double)o[0] + (double)o[1]) + ((double)o[2] + (double)o[3]);
        }
    }
    if (a.last) {
        const double t = block_sum_fixed<NT>(part, red);
        if (threadIdx.x == 0) a.partials[(size_t)sample * a.tiles + tile] = t;
    }
}

template <int R, int RY, int TXT, int TYT>
constexpr size_t tile_smem_bytes() {
    return (size_t)(RY * TYT + 2 * R) * (4 * TXT + 2 * ((R + 3) & ~3)) * sizeof(float);
}

// Whole field resident in shared memory for every step (one CTA per sample).  The
// padded array holds the n x n field plus its periodic images in an R-row / R4-column
// collar.  Each step every thread computes its 4 x RY block into registers, the block
// synchronises, and the new values are written over the old ones and their images.
struct ResidentArgs {
    const float *u0;
    float *uT;
    const StepCoef *coef;
    double *ubar;
    double *ooi;
    const int *steps_ps;  // per-sample step counts (serving), or nullptr: nsteps for all
    int n;
    int ns;
    int nsteps;
};

template <int R, int RY>
__global__ void __launch_bounds__(256) resident_kernel(ResidentArgs a) {
    constexpr int RX = 4;
    constexpr int R4 = (R + 3) & ~3;
    constexpr int WIN = RX + 2 * R4;
    constexpr DiscRows<R> disc{};
    extern __shared__ float4 smem4[];
    float *s = reinterpret_cast<float *>(smem4);
    __shared__ double red[256];

    const int n = a.n;
    const int SW = n + 2 * R4;
    const int SW4 = SW / 4;
    const int SH = n + 2 * R;
    const int TXT = n / 4;
    const int tx = threadIdx.x % TXT;
    const int ty = threadIdx.x / TXT;
    const int ox = tx * RX;
    const int oy = ty * RY;
    const int nt = blockDim.x;
    const size_t nn = (size_t)n * n;

    for (int sample = blockIdx.x; sample < a.ns; sample += gridDim.x) {
        const float *__restrict__ src = a.u0 + (size_t)sample * nn;
        for (int idx = threadIdx.x; idx < SH * SW4; idx += nt) {
            const int r = idx / SW4;
            const int c4 = idx - r * SW4;
            const int gy = wrap_idx(r - R, n);
            const int gx = wrap_idx(4 * c4 - R4, n);
            smem4[idx] = __ldg(reinterpret_cast<const float4 *>(src + (size_t)gy * n + gx));
        }
        const StepCoef cf = a.coef[sample];
        __syncthreads();

        float o[RY][RX];
        const int nsteps = a.steps_ps ? a.steps_ps[sample] : a.nsteps;
        for (int step = 0; step < nsteps; ++step) {
            float acc[RY][RX];
#pragma unroll
            for (int j = 0; j < RY; ++j)
#pragma unroll
                for (int i = 0; i < RX; ++i) acc[j][i] = 0.f;
#pragma unroll
            for (int r = 0; r < RY + 2 * R; ++r) {
                const float4 *rowp = reinterpret_cast<const float4 *>(s + (oy + r) * SW + ox);
                float v[WIN];
#pragma unroll
                for (int q = 0; q < WIN / 4; ++q) {
                    const float4 t = rowp[q];
                    v[4 * q + 0] = t.x;
                    v[4 * q + 1] = t.y;
                    v[4 * q + 2] = t.z;
                    v[4 * q + 3] = t.w;
                }
                float p[RX + 2 * R + 1];
                p[0] = 0.f;
#pragma unroll
                for (int k = 0; k < RX + 2 * R; ++k) p[k + 1] = p[k] + v[R4 - R + k];
#pragma unroll
                for (int j = 0; j < RY; ++j) {
                    const int dy = r - R - j;
                    if (dy >= -R && dy <= R) {
                        const int w = disc.w[dy < 0 ? -dy : dy];
#pragma unroll
                        for (int i = 0; i < RX; ++i) acc[j][i] += p[i + R + w + 1] - p[i + R - w];
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < RY; ++j) {
                const float4 c4v = *reinterpret_cast<const float4 *>(s + (oy + j + R) * SW + ox + R4);
                const float uc[4] = {c4v.x, c4v.y, c4v.z, c4v.w};
#pragma unroll
                for (int i = 0; i < RX; ++i) {
                    const float sd = fmaf(-cf.c0, uc[i], acc[j][i]);
                    const float v = uc[i] + fmaf(cf.c1, sd, cf.c2 * uc[i]);
                    o[j][i] = fminf(1.f, fmaxf(-1.f, v));
                }
            }
            __syncthreads();
            // write back the block and its periodic images
            const bool left = ox < R4, right = ox >= n - R4;
#pragma unroll
            for (int j = 0; j < RY; ++j) {
                const float4 val = make_float4(o[j][0], o[j][1], o[j][2], o[j][3]);
                const int y = oy + j;
                const int rows[3] = {y + R, y < R ? y + R + n : -1, y >= n - R ? y + R - n : -1};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int pr = rows[q];
                    if (pr < 0) continue;
                    float *rowb = s + pr * SW;
                    *reinterpret_cast<float4 *>(rowb + ox + R4) = val;
                    if (left) *reinterpret_cast<float4 *>(rowb + ox + R4 + n) = val;
                    if (right) *reinterpret_cast<float4 *>(rowb + ox + R4 - n) = val;
                }
            }
            __syncthreads();
        }
        // output of interest and optional final field
        double part = 0.0;
#pragma unroll
        for (int j = 0; j < RY; ++j) {
            const float4 c4v = *reinterpret_cast<const float4 *>(s + (oy + j + R) * SW + ox + R4);
            part += ((double)c4v.x + (double)c4v.y) + ((double)c4v.z + (double)c4v.w);
            if (a.uT)
                *reinterpret_cast<float4 *>(a.uT + (size_t)sample * nn + (size_t)(oy + j) * n + ox) = c4v;
        }
        red[threadIdx.x] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < nt; ++i) t += red[i];
            const double mean = t / (double)nn;
            if (a.ubar) a.ubar[sample] = mean;
            if (a.ooi) a.ooi[sample] = 0.5 * (1.0 + mean);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- launchers
// Register-tiled kernel configuration per R: 64-column tiles, 4 x RY outputs per thread.
template <int R>
struct TileCfg {
    static constexpr int RY = R <= 4 ? 8 : 16;
    static constexpr int TXT = 16;
    static constexpr int TYT = 8;
    static constexpr int TX = 4 * TXT;
    static constexpr int TY = RY * TYT;
};

template <int R, int ALGO>
mfmc_status launch_tile(const TileArgs &base, size_t ns, cudaStream_t st) {
    using C = TileCfg<R>;
    auto kern = step_tile_kernel<R, C::RY, C::TXT, C::TYT, ALGO>;
    constexpr size_t smem = tile_smem_bytes<R, C::RY, C::TXT, C::TYT>();
    // set before every launch: the attribute is per device, and the call is cheap
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (size_t s0 = 0; s0 < ns; s0 += 65535) {
        TileArgs a = base;
        a.sample0 = (int)s0;
        const unsigned gy = (unsigned)(ns - s0 < 65535 ? ns - s0 : 65535);
        kern<<<dim3(a.tiles, gy), C::TXT * C::TYT, smem, st>>>(a);
    }
    MFMC_LAUNCHED("step_kernels launch 1");
    return MFMC_OK;
}

struct TileLauncher {
    int tx, ty;
    mfmc_status (*fn[3])(const TileArgs &, size_t, cudaStream_t);  // direct, prefix, prefix-Kahan
};

template <int R, bool DIRECT>
TileLauncher make_tile_launcher() {
    TileLauncher L;
    L.tx = TileCfg<R>::TX;
    L.ty = TileCfg<R>::TY;
    if constexpr (DIRECT) {
        L.fn[0] = &launch_tile<R, 0>;
    } else {
        L.fn[0] = nullptr;
    }
    L.fn[1] = &launch_tile<R, 1>;
    L.fn[2] = nullptr;  // the compensated form runs on the TMA pipeline
    return L;
}

constexpr int RES_RY = 16;

inline size_t resident_smem(int n, int R) {
    const int R4 = (R + 3) & ~3;
    return (size_t)(n + 2 * R) * (n + 2 * R4) * sizeof(float);
}

inline int resident_threads(int n) { return n * n / (4 * RES_RY); }

template <int R>
mfmc_status launch_resident(const ResidentArgs &a, cudaStream_t st) {
    auto kern = resident_kernel<R, RES_RY>;
    const size_t smem = resident_smem(a.n, R);
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nt = resident_threads(a.n);
    int per_sm = 0;
    MFMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
    int dev = 0, sms = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int cap = (per_sm > 0 ? per_sm : 1) * sms;
    const int grid = a.ns < cap ? a.ns : cap;
    kern<<<grid > 0 ? grid : 1, nt, smem, st>>>(a);
    MFMC_LAUNCHED("step_kernels launch 2");
    return MFMC_OK;
}

typedef mfmc_status (*ResidentFn)(const ResidentArgs &, cudaStream_t);

// Defined in the per-R translation units.
const TileLauncher *tile_launcher(int R);
ResidentFn resident_launcher(int R);

}  // namespace mfmc
