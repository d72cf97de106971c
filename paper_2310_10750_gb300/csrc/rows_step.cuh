// Row-streaming step kernel (constant kernel, R <= 12).
//
// A work item is a band of BH lattice rows of one sample, across the full width: thread t
// owns the four columns 4t .. 4t+3 (n/4 threads) and walks down the band's BH + 2R input
// rows once.  Each input row is loaded (float4) from a ring of shared-memory chunks that
// TMA fills from the ghost-framed field (chunks of CH >= R rows, NCH stages, the copy of a
// chunk two ahead in flight while the current one is read).  From the row the thread
// forms an in-register prefix sum, one segment sum per distinct disc-row half-width, and
// adds each to the 2R+1 outputs that row touches; the accumulators form a ring of 2R+1
// slots, so after row q the output q - 2R is complete and is finished (update, projection,
// store with ghost images, OoI partial at the last step).  Unrolling the row loop by the
// ring period 2R+1 keeps every slot index static.  Every halo row is summed once per band
// instead of once per output block, which is what makes this cheaper than the tile
// kernels: about 2R+1 + (4+2R+4 w)/4 * (BH+2R)/BH + 5 FP32 instructions per point,
// w = number of distinct half-widths.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tma_step.cuh"

namespace mfmc {

struct RowsArgs {
    float *dst;            // padded destination (nullptr: no field output)
    float *dst_plain;      // unpadded destination at the last step, or nullptr
    const StepCoef *coef;
    double *partials;      // [ns][bands]
    int *status;
    const int *steps_ps;   // per-sample step counts, or nullptr
    int step;
    int n, P, BW, nbox, BH, bands, total, last;
};

template <int R, int RX>
struct RowsCfg {
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int CH = R < 8 ? 8 : R;  // chunk rows; >= R so a chunk two back is free
    static constexpr int NCH = 4;              // ring stages
    static constexpr int PER = 2 * R + 1;      // accumulator ring period
    static constexpr int WIN = RX + 2 * R4;    // floats a thread reads per row
};

// RX consecutive floats (RX = 2 or 4) from shared memory.
template <int RX>
__device__ __forceinline__ void load_vec(const float *p, float *out) {
    if constexpr (RX == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        out[0] = x.x;
        out[1] = x.y;
        out[2] = x.z;
        out[3] = x.w;
    } else {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        out[0] = x.x;
        out[1] = x.y;
    }
}

template <int RX>
__device__ __forceinline__ void store_vec(float *p, const float *v) {
    if constexpr (RX == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
}

// RX: columns per thread (4, or 2 for twice the threads at ~12 % more adds per point).
template <int R, int RX>
__global__ void __launch_bounds__(512) step_rows_kernel(const __grid_constant__ CUtensorMap map, RowsArgs a) {
    using C = RowsCfg<R, RX>;
    constexpr int CH = C::CH, NCH = C::NCH, PER = C::PER, WIN = C::WIN, R4 = C::R4;
    constexpr DiscRows<R> disc{};
    extern __shared__ unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NCH];
    __shared__ double red[16];
    __shared__ int abort_flag;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = a.n, G = R4;
    const int stage_floats = CH * a.BW * a.nbox;
    const uint32_t chunk_bytes = (uint32_t)stage_floats * sizeof(float);
    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();

    // offsets (within a chunk's row 0) of this thread's WIN/RX vectors of a row: padded
    // columns RX tid + RX q, boxes laid out one after the other, each [CH][BW]
    int off[WIN / RX];
#pragma unroll
    for (int q = 0; q < WIN / RX; ++q) {
        const int col = RX * tid + RX * q;
        off[q] = (col / a.BW) * (CH * a.BW) + (col % a.BW);
    }
    const int coff = ((RX * tid + R4) / a.BW) * (CH * a.BW) + ((RX * tid + R4) % a.BW);  // centre vector

    uint32_t gchunk = 0;  // chunks consumed by this CTA so far (ring position and barrier phase)
    const int rows = a.BH + 2 * R;
    const int nchunks = (rows + CH - 1) / CH;

    for (int item = blockIdx.x; item < a.total; item += gridDim.x) {
        const int sample = item / a.bands, band = item - sample * a.bands;
        if (a.steps_ps != nullptr && a.step > a.steps_ps[sample]) continue;
        const bool last = a.last || (a.steps_ps != nullptr && a.step == a.steps_ps[sample]);
        const int y0 = band * a.BH;
        auto issue = [&](int c) {
            const uint32_t g = gchunk + c;
            const int st = g % NCH;
            float *dstc = ring + st * stage_floats;
            mbar_expect_tx(&full[st], chunk_bytes);
            for (int b = 0; b < a.nbox; ++b)
                tma_load_3d(dstc + b * CH * a.BW, &map, &full[st], b * a.BW, G + y0 - R + c * CH, sample);
        };
        if (tid == 0)
            for (int c = 0; c < NCH - 2 && c < nchunks; ++c) issue(c);

        float acc[PER][RX];
#pragma unroll
        for (int k = 0; k < PER; ++k)
#pragma unroll
            for (int i = 0; i < RX; ++i) acc[k][i] = 0.f;
        const StepCoef cf = a.coef[sample];
        double part = 0.0;
        bool aborted = false;

        for (int q0 = 0; q0 < rows; q0 += PER) {
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                const int q = q0 + m;
                if (q < rows) {
                    if (q % CH == 0) {
                        const int c = q / CH;
                        __syncthreads();  // every thread is past chunk c-1: chunk c-2 is free
                        if (tid == 0 && c + NCH - 2 < nchunks) issue(c + NCH - 2);
                        const uint32_t g = gchunk + c;
                        long long spins = 0;
                        while (!mbar_try_wait(&full[g % NCH], (g / NCH) & 1)) {
                            if (++spins > kWaitLimit) {
                                abort_flag = 1;
                                break;
                            }
                        }
                        __syncthreads();
                        if (abort_flag) {
                            aborted = true;
                            break;
                        }
                    }
                    const float *rowp = ring + ((gchunk + q / CH) % NCH) * stage_floats + (q % CH) * a.BW;
                    float v[WIN];
#pragma unroll
                    for (int t = 0; t < WIN / RX; ++t) load_vec<RX>(rowp + off[t], v + RX * t);
                    float p[RX + 2 * R + 1];
                    p[0] = 0.f;
#pragma unroll
                    for (int k = 0; k < RX + 2 * R; ++k) p[k + 1] = p[k] + v[R4 - R + k];
                    // row q adds to outputs q - 2R + kk, kk = 0..2R, with dy = R - kk
#pragma unroll
                    for (int kk = 0; kk < PER; ++kk) {
                        const int dyy = R - kk;
                        const int w = disc.w[dyy < 0 ? -dyy : dyy];
                        const int slot = (m + kk + 1) % PER;
#pragma unroll
                        for (int i = 0; i < RX; ++i) acc[slot][i] += p[i + R + w + 1] - p[i + R - w];
                    }
                    // output o = q - 2R is complete
                    const int o = q - 2 * R;
                    const int slot0 = (m + 1) % PER;
                    if (o >= 0) {
                        const int qc = o + R;  // its centre row
                        float uc[RX];
                        load_vec<RX>(ring + ((gchunk + qc / CH) % NCH) * stage_floats + (qc % CH) * a.BW + coff, uc);
                        float out[RX];
#pragma unroll
                        for (int i = 0; i < RX; ++i) {
                            const float sd = fmaf(-cf.c0, uc[i], acc[slot0][i]);
                            const float vv = uc[i] + fmaf(cf.c1, sd, cf.c2 * uc[i]);
                            out[i] = fminf(1.f, fmaxf(-1.f, vv));
                        }
                        const int y = y0 + o, x = RX * tid;
                        if (y < n) {
                            if (a.dst_plain) {
                                store_vec<RX>(a.dst_plain + (size_t)sample * n * n + (size_t)y * n + x, out);
                            } else if (a.dst) {
                                float *d = a.dst + (size_t)sample * a.P * a.P;
                                const int rws[3] = {G + y, y < G ? G + y + n : -1, y >= n - G ? G + y - n : -1};
                                const int cls[3] = {G + x, x < G ? G + x + n : -1, x >= n - G ? G + x - n : -1};
#pragma unroll
                                for (int r2 = 0; r2 < 3; ++r2) {
                                    if (rws[r2] < 0) continue;
#pragma unroll
                                    for (int c2 = 0; c2 < 3; ++c2) {
                                        if (cls[c2] < 0) continue;
                                        store_vec<RX>(d + (size_t)rws[r2] * a.P + cls[c2], out);
                                    }
                                }
                            }
                            if (last) {
                                if constexpr (RX == 4)
                                    part += ((double)out[0] + (double)out[1]) + ((double)out[2] + (double)out[3]);
                                else
                                    part += (double)out[0] + (double)out[1];
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < RX; ++i) acc[slot0][i] = 0.f;
                }
            }
            if (aborted) break;
        }
        if (aborted) {
            if (tid == 0) atomicExch(a.status, 1);
            break;
        }
        gchunk += nchunks;
        if (last) {
            for (int off2 = 16; off2 > 0; off2 >>= 1) part += __shfl_down_sync(0xffffffffu, part, off2);
            if ((tid & 31) == 0) red[tid >> 5] = part;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int i = 0; i < (nt + 31) / 32; ++i) t += red[i];
                a.partials[(size_t)sample * a.bands + band] = t;
            }
        }
        __syncthreads();  // the ring is reused by the next item
    }
}

struct RowsLauncher {
    int ch;  // chunk rows (TMA box height)
    // [0]: 4 columns per thread, [1]: 2 columns per thread
    mfmc_status (*fn[2])(const CUtensorMap &, const RowsArgs &, int grid, int threads, size_t smem, cudaStream_t);
    int (*blocks_per_sm[2])(int threads, size_t smem);
};

template <int R, int RX>
mfmc_status launch_rows(const CUtensorMap &map, const RowsArgs &a, int grid, int threads, size_t smem,
                        cudaStream_t st) {
    auto kern = step_rows_kernel<R, RX>;
    static size_t attr = 0;
    if (smem > attr) {
        MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    kern<<<grid, threads, smem, st>>>(map, a);
    MFMC_LAUNCHED("rows_step launch");
    return MFMC_OK;
}

template <int R, int RX>
int rows_blocks_per_sm(int threads, size_t smem) {
    auto kern = step_rows_kernel<R, RX>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    (void)cudaGetLastError();  // a failed query must not be reported by a later launch check
    return e == cudaSuccess && per > 0 ? per : 1;
}

template <int R>
RowsLauncher make_rows_launcher() {
    RowsLauncher L;
    L.ch = RowsCfg<R, 4>::CH;
    L.fn[0] = &launch_rows<R, 4>;
    L.fn[1] = &launch_rows<R, 2>;
    L.blocks_per_sm[0] = &rows_blocks_per_sm<R, 4>;
    L.blocks_per_sm[1] = &rows_blocks_per_sm<R, 2>;
    return L;
}

// Defined in the per-R translation units (R <= 12).
const RowsLauncher *rows_launcher(int R);

}  // namespace mfmc
