// Spectral step on this library's own FFT kernels (MFMC_ALGO_SPECTRAL): n = 1024 here, n = 64 and
// 128 in the resident register-transform form below, other even n <= 128 in the resident
// mixed-radix form (spectral_resident.cu).
//
// On the periodic lattice the nodal quadrature (gamma * u)_i = sum_{z in D} w_z u_{i+z}
// (Section 2) is a circular convolution, so S = IFFT2(FFT2(u) * K^) with K^ the transform of
// the disc weights; the disc is symmetric under z -> -z, so K^ is real.  Its cost per point does
// not depend on the horizon, which makes it the fast form for the large horizons (delta = 32h:
// 3209 disc points).  A time step is two kernels:
//
//   column pass   for each half-spectrum column kx of each sample: forward FFT over y,
//                 product with K^(ky, kx) / n^2, inverse FFT over y (the column never leaves
//                 shared memory between the two transforms);
//   row pass      for each pair of rows (y, y + 1) of each sample: the inverse row transform
//                 of the two half-spectrum rows packed as one complex sequence gives S on both
//                 rows (real and imaginary part), the update of Eq. nonl_CH_nm with beta2 = 0
//                 and the projection of Eq. potential_obstacle give the new rows, which are
//                 stored and at once transformed forward (again packed in pairs) into the
//                 half-spectrum rows of the next step.
//
// A 1024-point transform is done by one warp as 32 x 32 (four-step): each lane transforms 32
// values in registers (radix-2, decimation in frequency), multiplies by W_1024^(t k), and a
// skewed transpose through shared memory hands every lane one column of the 32 x 32 array for
// the second 32-point transform.  Forward transforms are unnormalised; 1 / n^2 is folded into K^.
// The half spectrum is stored [sample][ky][kx] with kx = 0..512 in a row of 528 complex values.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "mfmc_internal.h"
#include "spectral_queue.cuh"
#include "tma_step.cuh"

namespace mfmc {

namespace {
constexpr int kSq = 32;               // n = kSq * kSq
constexpr int kN = kSq * kSq;         // 1024
constexpr int kHalf = kN / 2 + 1;     // 513 half-spectrum columns
constexpr int kColTile = 8;           // columns per column-pass CTA (one warp each)
constexpr int kPitch = 528;           // half-spectrum row pitch in complex values: 66 tiles of 8
constexpr int kColStride = kColTile + 1;  // shared-memory row stride of a column tile (complex)
constexpr int kRowWarps = 12;         // row-pass warps per CTA
constexpr int kSpecRowBytes = 514 * 8;    // a half-spectrum row as copied (513 values and one of padding)
constexpr int kRowBuf = 2 * 514;      // a row-pass warp buffer in complex values (8224 bytes)
}  // namespace

// exp(-2 pi i k / 32), k = 0..31, written once per device from the host (FP64 sin and cos)
__constant__ float2 c_w32[kSq];

// complex sums as packed FP32 pairs (each half rounds exactly like the scalar operation)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one packed instruction, rounded once like the scalar subtraction
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// a * w, or a * conj(w) for the inverse transform
template <bool INV>
__device__ __forceinline__ float2 cmulw(float2 a, float2 w) {
    if (INV) return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -(a.x * w.y)));
    return make_float2(fmaf(a.x, w.x, -(a.y * w.y)), fmaf(a.x, w.y, a.y * w.x));
}

__host__ __device__ constexpr int brev5(int k) {
    return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

// In-register 32-point FFT: radix-2 decimation in frequency, natural order in, bit-reversed
// order out (X[k] in v[brev5(k)]).  Every index and twiddle exponent is static after unrolling.
template <bool INV>
__device__ __forceinline__ void fft32(float2 (&v)[kSq]) {
#pragma unroll
    for (int span = kSq / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int g = 0; g < kSq; g += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const float2 a = v[g + j], b = v[g + j + span];
                v[g + j] = cadd(a, b);
                const float2 d = csub(a, b);
                const int e = j * (kSq / (2 * span));  // twiddle W_32^e
                if (e == 0)
                    v[g + j + span] = d;
                else if (e == kSq / 4)  // W_32^8 = -i (its conjugate: +i)
                    v[g + j + span] = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                else
                    v[g + j + span] = cmulw<INV>(d, c_w32[e]);
            }
        }
    }
}

// 1024-point FFT by one warp (four-step, 32 x 32).  On entry lane t holds x[t + 32 j] in v[j];
// on return X[t + 32 j] in v[j].  scr: 1024 complex of scratch, element p at scr[p * STRIDE];
// tw: W_1024^(t k) at tw[k * 32 + t].
template <bool INV, int STRIDE>
__device__ __forceinline__ void warp_fft1024(float2 (&v)[kSq], float2 *scr, const float2 *tw, int t) {
    fft32<INV>(v);  // Y[t][k2] = sum_j x[t + 32 j] W_32^(j k2), in v[brev5(k2)]
    // Y[t][k2] W_1024^(t k2) into row k2, column t of the 32 x 32 array, stored with column
    // (t + k2) mod 32 so that both the row writes and the column reads are conflict-free
#pragma unroll
    for (int k2 = 0; k2 < kSq; ++k2)
        scr[(k2 * kSq + ((t + k2) & 31)) * STRIDE] = cmulw<INV>(v[brev5(k2)], tw[k2 * kSq + t]);
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < kSq; ++n1) v[n1] = scr[(t * kSq + ((n1 + t) & 31)) * STRIDE];  // Y[n1][t]
    __syncwarp();
    fft32<INV>(v);  // X[t + 32 k1] = sum_n1 Y[n1][t] W_1024^(n1 t) W_32^(n1 k1), in v[brev5(k1)]
    float2 o[kSq];
#pragma unroll
    for (int k = 0; k < kSq; ++k) o[k] = v[brev5(k)];
#pragma unroll
    for (int k = 0; k < kSq; ++k) v[k] = o[k];
}

// Column pass: CTA (tile, sample) transforms columns kx = 8 tile .. 8 tile + 7 of the sample's
// half spectrum over y, multiplies by khatT[kx][ky] (K^(ky, kx) / n^2 in both halves of a pair)
// and transforms back.
// One warp per column; the tile arrives by asynchronous 8-byte copies into rows of 9 complex
// values (conflict-free column access) and stays in shared memory; two CTAs per SM overlap one
// tile's copies with the other's transforms.
__global__ void __launch_bounds__(kColTile * 32, 2)
    spectral_column_kernel(float2 *spec, const float2 *khatT, const float2 *twg) {
    extern __shared__ float2 spec_smem[];
    float2 *tile = spec_smem;                    // [1024][9]
    float2 *tw = spec_smem + kN * kColStride;    // [32][32]
    const int ti = blockIdx.x;
    float2 *g = spec + (size_t)blockIdx.y * kN * kPitch + ti * kColTile;
    for (int i = threadIdx.x; i < kN * kColTile; i += blockDim.x) {
        const int y = i / kColTile, c = i - y * kColTile;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(tile + y * kColStride + c)),
                     "l"(g + (size_t)y * kPitch + c)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int i = threadIdx.x; i < kSq * kSq; i += blockDim.x) tw[i] = twg[i];
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31, kx = ti * kColTile + w;
    if (kx < kHalf) {
        float2 *col = tile + w;  // element y at col[y * kColStride]
        float2 v[kSq];
#pragma unroll
        for (int j = 0; j < kSq; ++j) v[j] = col[(t + kSq * j) * kColStride];
        __syncwarp();
        warp_fft1024<false, kColStride>(v, col, tw, t);
        const float2 *kh = khatT + (size_t)kx * kN;
#pragma unroll
        for (int j = 0; j < kSq; ++j) v[j] = __fmul2_rn(v[j], __ldg(kh + t + kSq * j));
        warp_fft1024<true, kColStride>(v, col, tw, t);
#pragma unroll
        for (int j = 0; j < kSq; ++j) col[(t + kSq * j) * kColStride] = v[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kN * kColTile; i += blockDim.x) {
        const int y = i / kColTile, c = i - y * kColTile;
        g[(size_t)y * kPitch + c] = tile[y * kColStride + c];
    }
}

// 1-D bulk copy global -> shared of `bytes` (a multiple of 16, both addresses 16-byte aligned),
// completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of a warp's barrier (all lanes); false when it gave up.
__device__ __forceinline__ bool spec_wait(uint64_t *bar, uint32_t parity) {
    long long spins = 0;
    while (!mbar_try_wait(bar, parity))
        if (++spins > kWaitLimit) return false;
    return true;
}

// Row pass over the row pairs (y, y + 1) of every sample, one warp per pair at a time.
//   UPDATE: the pair's half-spectrum rows A (row y) and B (row y + 1) of the product are
//     combined into Z[k] = A[k] + i B[k] for k = 0..1023 (A[k] = conj(A[n - k]) above n/2),
//     whose inverse transform is S_y + i S_{y+1}; the update and projection of the rows of
//     `src` are stored to `dst`.
//   FWD: the pair of new rows (or, without UPDATE, of `src`) as one complex row, its forward
//     transform Z, and the half spectra A[k] = (Z[k] + conj(Z[n-k])) / 2,
//     B[k] = (Z[k] - conj(Z[n-k])) / 2i, k = 0..512, stored for the next column pass.
// Each warp owns two shared buffers of 8224 bytes fed by bulk copies: with UPDATE one holds the
// pair's spectrum rows (and then serves as the transforms' scratch), the other its rows of
// `src`; the copies for the next pair go into each buffer as soon as it is free, so they are in
// flight during this pair's transforms, and the roles swap from pair to pair.  Without UPDATE
// the two buffers take the rows of `src` of alternate pairs.
template <bool UPDATE, bool FWD>
__global__ void __launch_bounds__(kRowWarps * 32, 1)
    spectral_row_kernel(float2 *spec, const float *src, float *dst, const StepCoef *coef, const float2 *twg,
                        long long pairs, int *status) {
    extern __shared__ __align__(16) float2 spec_smem[];
    __shared__ __align__(8) uint64_t bars[kRowWarps][2];
    float2 *tw = spec_smem;
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    float2 *const buf0 = spec_smem + kSq * kSq + 2 * w * kRowBuf;  // buffer b at buf0 + b kRowBuf
    auto buf = [&](int b) { return buf0 + b * kRowBuf; };
    uint64_t *bar = bars[w];
    for (int i = threadIdx.x; i < kSq * kSq; i += blockDim.x) tw[i] = twg[i];
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * kRowWarps;
    long long p = (long long)blockIdx.x * kRowWarps + w;
    uint32_t phases = 0u;  // bit b: the parity of the next completion of barrier b
    // the copies of pair q: its spectrum rows (2 x 514 complex) and its rows of src (8 KB)
    auto load_spec = [&](long long q, int b) {
        if (t == 0) {
            const long long smp = q / (kN / 2);
            const int y = 2 * (int)(q - smp * (kN / 2));
            const float2 *sa = spec + ((size_t)smp * kN + y) * kPitch;
            mbar_expect_tx(&bar[b], 2 * kSpecRowBytes);
            bulk_load(buf(b), sa, kSpecRowBytes, &bar[b]);
            bulk_load(buf(b) + kSpecRowBytes / 8, sa + kPitch, kSpecRowBytes, &bar[b]);
        }
    };
    auto load_rows = [&](long long q, int b) {
        if (t == 0) {
            const long long smp = q / (kN / 2);
            const int y = 2 * (int)(q - smp * (kN / 2));
            mbar_expect_tx(&bar[b], 2 * kN * sizeof(float));
            bulk_load(buf(b), src + ((size_t)smp * kN + y) * kN, 2 * kN * sizeof(float), &bar[b]);
        }
    };
    // a buffer is refilled only after every lane has read it (the generic-proxy reads are
    // ordered before the copy's writes)
    auto release = [&]() {
        __syncwarp();
        if (t == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    int sb = 0, ub = 1;  // UPDATE: buffer of the spectrum rows, of the rows of src
    if (p < pairs) {
        if (UPDATE) {
            load_spec(p, sb);
            load_rows(p, ub);
        } else {
            load_rows(p, 0);
        }
    }
    for (int it = 0; p < pairs; p += stride, ++it) {
        const long long smp = p / (kN / 2);
        const int y = 2 * (int)(p - smp * (kN / 2));
        const long long nxt = p + stride;
        float2 v[kSq];
        if (UPDATE) {
            if (!spec_wait(&bar[sb], (phases >> sb) & 1u)) goto timeout;
            phases ^= 1u << sb;
            {
                const float2 *A = buf(sb), *B = buf(sb) + kSpecRowBytes / 8;
#pragma unroll
                for (int j = 0; j < kSq; ++j) {
                    const int k = t + kSq * j;
                    if (k <= kN / 2) {
                        const float2 a = A[k], b = B[k];
                        v[j] = make_float2(a.x - b.y, a.y + b.x);
                    } else {
                        const float2 a = A[kN - k], b = B[kN - k];
                        v[j] = make_float2(a.x + b.y, b.x - a.y);
                    }
                }
            }
            __syncwarp();
            warp_fft1024<true, 1>(v, buf(sb), tw, t);  // S_y + i S_{y+1} at x = t + 32 j
            if (!FWD) {
                release();
                if (nxt < pairs) load_rows(nxt, sb);
            }
            if (!spec_wait(&bar[ub], (phases >> ub) & 1u)) goto timeout;
            phases ^= 1u << ub;
            {
                const StepCoef cf = coef[smp];
                const float *U = reinterpret_cast<const float *>(buf(ub));
                float *da = dst + ((size_t)smp * kN + y) * kN, *db = da + kN;
#pragma unroll
                for (int j = 0; j < kSq; ++j) {
                    const int x = t + kSq * j;
                    const float u0 = U[x], u1 = U[kN + x];
                    const float v0 = u0 + fmaf(cf.c1, fmaf(-cf.c0, u0, v[j].x), cf.c2 * u0);
                    const float v1 = u1 + fmaf(cf.c1, fmaf(-cf.c0, u1, v[j].y), cf.c2 * u1);
                    const float n0 = fminf(1.f, fmaxf(-1.f, v0)), n1 = fminf(1.f, fmaxf(-1.f, v1));
                    da[x] = n0;
                    db[x] = n1;
                    v[j] = make_float2(n0, n1);
                }
            }
            release();
            if (nxt < pairs) load_spec(nxt, ub);
        } else {
            const int b = it & 1;
            if (nxt < pairs) load_rows(nxt, b ^ 1);
            if (!spec_wait(&bar[b], (phases >> b) & 1u)) goto timeout;
            phases ^= 1u << b;
            const float *U = reinterpret_cast<const float *>(buf(b));
#pragma unroll
            for (int j = 0; j < kSq; ++j) v[j] = make_float2(U[t + kSq * j], U[kN + t + kSq * j]);
            __syncwarp();
            sb = b;  // the transform's scratch
        }
        if (FWD) {
            warp_fft1024<false, 1>(v, buf(sb), tw, t);
            float2 *scr = buf(sb);
#pragma unroll
            for (int j = 0; j < kSq; ++j) scr[t + kSq * j] = v[j];
            __syncwarp();
            float2 *sa = spec + ((size_t)smp * kN + y) * kPitch, *sbp = sa + kPitch;
#pragma unroll
            for (int j = 0; j <= kN / 2 / kSq; ++j) {
                const int k = t + kSq * j;
                if (k <= kN / 2) {
                    const float2 zk = scr[k], zm = scr[(kN - k) & (kN - 1)];
                    sa[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    sbp[k] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
                }
            }
            if (UPDATE) {
                release();
                if (nxt < pairs) load_rows(nxt, sb);
            } else {
                release();
            }
        }
        if (UPDATE) {
            const int tmp = sb;
            sb = ub;
            ub = tmp;
        }
    }
    return;
timeout:
    // a copy that never lands: report, then wait (again bounded) for the warp's other copy in
    // flight so that no copy targets the buffers after the CTA exits
    if (t == 0) {
        atomicExch(status, 1);
        for (int b = 0; b < 2; ++b) {
            long long spins = 0;
            while (!mbar_try_wait(&bar[b], (phases >> b) & 1u) && ++spins < kWaitLimit) {
            }
        }
    }
}

// ----------------------------------------------------------------------------- small lattices
// n = 32 E with E = 2 or 4 (n = 64, 128: the paper's meshes h = 1/64 and 1/128): a CTA keeps its
// samples' fields and half spectra in shared memory for every step (one sample at n = 128, four
// at n = 64) and writes only the final fields and their OoI.  A warp transforms 32 / E
// sequences of length n at once, E lanes each: every lane transforms its 32 values (stride E)
// in registers, multiplies by W_n^(n1 k2), and after an exchange through the warp's scratch
// takes E-point DFTs across the E lanes (four-step with n = E x 32).
template <int E>
struct SmallCfg {
    static constexpr int N = 32 * E, NH = N / 2 + 1;
    static constexpr int F = 32 / E;                         // transforms per warp
    static constexpr int Q = 32 / E;                         // k2 values per lane after the exchange
    static constexpr int SPC = (128 / N) * (128 / N);        // samples per CTA
    static constexpr int WARPS = 9;                          // 8 for the row pairs, 9 for the columns
    // the field in rows of RS = N + 1 floats (the row pairs a warp transforms then start in
    // different banks), then the half spectrum (N RS is even: 8-byte aligned)
    static constexpr int RS = N + 1;
    static constexpr int SAMPLE_FLOATS = N * RS + 2 * N * NH;
    // a warp's scratch (complex values): the exchange of warp_fft_small (1024) and the forward
    // row pass's staging of its F transforms, each padded by one value (F (N + 1) >= 1024)
    static constexpr int SCR = F * (N + 1);
    static constexpr size_t SMEM = ((size_t)SPC * SAMPLE_FLOATS + 2 * (WARPS * SCR + E * 33)) * sizeof(float);
};

// E lanes per transform (lane t: transform f = t / E, n1 = t % E).  On entry lane (f, n1) holds
// x_f[n1 + E j] in v[j]; on return X_f[k2 + 32 k1] with k2 = n1 Q + q in v[q E + k1] (Q = 32 / E).
// scr: the warp's 1024 complex values of scratch; tw: W_n^(n1 k2) at tw[n1 * 33 + k2].
// The exchange stores element (f, k2, n1) in slot n1 ^ (k2 / Q) of its row of E, so that both
// the stores (fixed k2) and the loads (k2 = n1 Q + q, fixed q and m) touch every bank once.
template <int E, bool INV>
__device__ __forceinline__ void warp_fft_small(float2 (&v)[kSq], float2 *scr, const float2 *tw, int t) {
    constexpr int Q = 32 / E;
    const int f = t / E, n1 = t - f * E;
    fft32<INV>(v);  // Y_f[n1][k2] = sum_j x_f[n1 + E j] W_32^(j k2), in v[brev5(k2)]
    // Y_f[n1][k2] W_n^(n1 k2) to scratch element (32 f + ((k2 + f) mod 32)) E + (n1 ^ (k2 / Q))
#pragma unroll
    for (int k2 = 0; k2 < kSq; ++k2)
        scr[(f * kSq + ((k2 + f) & 31)) * E + (n1 ^ (k2 / Q))] = cmulw<INV>(v[brev5(k2)], tw[n1 * 33 + k2]);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k2 = n1 * Q + q;
        float2 y[E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[m] = scr[(f * kSq + ((k2 + f) & 31)) * E + (m ^ n1)];  // k2 / Q = n1
        if constexpr (E == 2) {
            v[q * 2 + 0] = cadd(y[0], y[1]);
            v[q * 2 + 1] = csub(y[0], y[1]);
        } else {  // E = 4: W_4 = -i (inverse: +i)
            const float2 s02 = cadd(y[0], y[2]), d02 = csub(y[0], y[2]);
            const float2 s13 = cadd(y[1], y[3]), d13 = csub(y[1], y[3]);
            const float2 r13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            v[q * 4 + 0] = cadd(s02, s13);
            v[q * 4 + 2] = csub(s02, s13);
            v[q * 4 + 1] = cadd(d02, r13);
            v[q * 4 + 3] = csub(d02, r13);
        }
    }
    __syncwarp();
}

// The whole solve of SPC samples per CTA on an n x n lattice, n = 32 E.  Per step: row pass
// (pairs of rows packed as one complex row, forward transform, split into the two half spectra),
// column pass (forward over y, product with khatT[kx][ky] = K^(ky, kx) / n^2, inverse), row pass
// (the two half-spectrum rows of a pair combined, inverse transform: S on both rows, update and
// projection in place).  Then the final fields to uT (when given) and the per-sample FP64 mean
// in a fixed order.  The samples s0 .. s0 + nloc - 1 (nloc <= SPC) by the CTA's C::WARPS warps;
// with STEPS, sample s takes steps_ps[s] steps (a sample whose steps are done keeps its field
// while the others go on), else every sample nsteps.  sm_small: C::SMEM bytes of shared memory;
// red: C::WARPS * 32 doubles.
template <int E, bool STEPS>
__device__ __forceinline__ void small_solve(const float *u0, float *uT, const StepCoef *coef, const float *khatT,
                                            const float2 *twg, int s0, int nloc, const int *steps_ps, int nsteps,
                                            double *ubar, double *ooi, float *sm_small, double *red) {
    using C = SmallCfg<E>;
    constexpr int N = C::N, NH = C::NH, F = C::F, Q = C::Q, SPC = C::SPC;
    float2 *scr_all = reinterpret_cast<float2 *>(sm_small + SPC * C::SAMPLE_FLOATS);
    float2 *tw = scr_all + C::WARPS * C::SCR;
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31, f = t / E, n1 = t - f * E;
    float2 *scr = scr_all + w * C::SCR;
    auto steps_of = [&](int s) { return s >= nloc ? 0 : steps_ps[s0 + s]; };
    int kmax = nsteps;
    if constexpr (STEPS) {
        kmax = 0;
        for (int s = 0; s < nloc; ++s) kmax = max(kmax, steps_of(s));
    }
    auto fld = [&](int s) { return sm_small + s * C::SAMPLE_FLOATS; };
    auto spc = [&](int s) { return reinterpret_cast<float2 *>(sm_small + s * C::SAMPLE_FLOATS + N * C::RS); };
    for (int i = threadIdx.x; i < SPC * N * N; i += blockDim.x) {
        const int s = i / (N * N), r = i - s * N * N;
        fld(s)[(r / N) * C::RS + r % N] = s < nloc ? u0[(size_t)(s0 + s) * N * N + r] : 0.f;
    }
    for (int i = threadIdx.x; i < E * 33; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    for (int step = 0; step < kmax; ++step) {
        if (w < 8) {  // forward row pass: pair p of the CTA's SPC * n / 2 pairs
            const int p = w * F + f, s = p / (N / 2), y = 2 * (p - s * (N / 2));
            const float *ua = fld(s) + y * C::RS, *ub = ua + C::RS;
            float2 v[kSq];
#pragma unroll
            for (int j = 0; j < kSq; ++j) v[j] = make_float2(ua[n1 + E * j], ub[n1 + E * j]);
            warp_fft_small<E, false>(v, scr, tw, t);
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k1 = 0; k1 < E; ++k1) scr[f * (N + 1) + n1 * Q + q + kSq * k1] = v[q * E + k1];
            __syncwarp();
            float2 *sa = spc(s) + y * NH, *sb = sa + NH;
#pragma unroll
            for (int i = 0; i <= N / 2 / E; ++i) {
                const int k = n1 + E * i;
                if (k <= N / 2) {
                    const float2 zk = scr[f * (N + 1) + k], zm = scr[f * (N + 1) + ((N - k) & (N - 1))];
                    sa[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    sb[k] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
                }
            }
            __syncwarp();
        }
        __syncthreads();
        {  // column pass: slot w + 9 f of the CTA's SPC * (n / 2 + 1) columns
            const int slot = w + C::WARPS * f;
            const bool active = slot < SPC * NH && slot / NH < nloc;
            const int sl = active ? slot : 0, s = sl / NH, c = sl - s * NH;
            float2 *col = spc(s) + c;  // element ky at col[ky * NH]
            float2 v[kSq];
#pragma unroll
            for (int j = 0; j < kSq; ++j) v[j] = col[(n1 + E * j) * NH];
            warp_fft_small<E, false>(v, scr, tw, t);
            const float *kh = khatT + (size_t)c * N;
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k1 = 0; k1 < E; ++k1) {
                    const int k = n1 * Q + q + kSq * k1;
                    const float kk = __ldg(kh + k);
                    if (active) col[k * NH] = make_float2(v[q * E + k1].x * kk, v[q * E + k1].y * kk);
                }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < kSq; ++j) v[j] = col[(n1 + E * j) * NH];
            warp_fft_small<E, true>(v, scr, tw, t);
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k1 = 0; k1 < E; ++k1)
                    if (active) col[(n1 * Q + q + kSq * k1) * NH] = v[q * E + k1];
        }
        __syncthreads();
        if (w < 8) {  // inverse row pass and the update
            const int p = w * F + f, s = p / (N / 2), y = 2 * (p - s * (N / 2));
            const float2 *sa = spc(s) + y * NH, *sb = sa + NH;
            float2 v[kSq];
#pragma unroll
            for (int j = 0; j < kSq; ++j) {
                const int k = n1 + E * j;
                if (k <= N / 2) {
                    const float2 a = sa[k], b = sb[k];
                    v[j] = make_float2(a.x - b.y, a.y + b.x);
                } else {
                    const float2 a = sa[N - k], b = sb[N - k];
                    v[j] = make_float2(a.x + b.y, b.x - a.y);
                }
            }
            warp_fft_small<E, true>(v, scr, tw, t);  // S_y + i S_{y+1} at x = n1 Q + q + 32 k1
            const StepCoef cf = coef[s0 + (s < nloc ? s : 0)];
            float *ua = fld(s) + y * C::RS, *ub = ua + C::RS;
            bool live = true;
            if constexpr (STEPS) live = step < steps_of(s);  // else the sample's steps are done
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k1 = 0; k1 < E; ++k1) {
                    const int x = n1 * Q + q + kSq * k1;
                    const float2 S = v[q * E + k1];
                    const float u0v = ua[x], u1v = ub[x];
                    const float v0 = u0v + fmaf(cf.c1, fmaf(-cf.c0, u0v, S.x), cf.c2 * u0v);
                    const float v1 = u1v + fmaf(cf.c1, fmaf(-cf.c0, u1v, S.y), cf.c2 * u1v);
                    if (live) {
                        ua[x] = fminf(1.f, fmaxf(-1.f, v0));
                        ub[x] = fminf(1.f, fmaxf(-1.f, v1));
                    }
                }
        }
        __syncthreads();
    }
    for (int s = 0; s < nloc; ++s) {
        const float *u = fld(s);
        double acc = 0.0;
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
            const float x = u[(i / N) * C::RS + i % N];
            acc += (double)x;
            if (uT) uT[(size_t)(s0 + s) * N * N + i] = x;
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < C::WARPS * 32; ++i) tot += red[i];
            const double mean = tot / ((double)N * N);
            if (ubar) ubar[s0 + s] = mean;
            if (ooi) ooi[s0 + s] = 0.5 * (1.0 + mean);
        }
        __syncthreads();
    }
}

template <int E>
__global__ void __launch_bounds__(SmallCfg<E>::WARPS * 32, 1)
    spectral_small_kernel(const float *u0, float *uT, const StepCoef *coef, const float *khatT, const float2 *twg,
                          int ns, int nsteps, double *ubar, double *ooi) {
    using C = SmallCfg<E>;
    extern __shared__ __align__(16) float sm_small[];
    __shared__ double red[C::WARPS * 32];
    const int s0 = blockIdx.x * C::SPC;
    const int nloc = ns - s0 < C::SPC ? ns - s0 : C::SPC;
    small_solve<E, false>(u0, uT, coef, khatT, twg, s0, nloc, nullptr, nsteps, ubar, ooi, sm_small, red);
}

// ----------------------------------------------------------------------------- the queue
// One sample's whole solve on the mixed-radix transforms (any even n <= 128 they serve): the
// field in shared memory, per step the disc sums of cta_disc_sums written straight into the
// update and projection (the pair's rows are no longer read by the transforms then), at the end
// the field to uT and the FP64 mean in a fixed order.  N > 0: n == N on the compile-time plan.
template <int N>
__device__ __noinline__ void sq_solve_generic(const SqModelDev &M, int s, float *smem, double *red) {
    const int n = M.plan.n, nn = n * n;
    float *u = smem;
    void *fsm = smem + nn;  // n even: n^2 floats keep the next region 16-byte aligned
    const float *src = M.u0 + (size_t)s * nn;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) u[i] = src[i];
    const StepCoef cf = M.coef[s];
    const int steps = M.steps_ps ? M.steps_ps[s] : M.nsteps;
    for (int k = 0; k < steps; ++k)
        cta_disc_sums<N, float>(
            M.plan, fsm, M.khat, M.tw, [&](int y, int x) { return u[y * n + x]; },
            [&](int y, int x, float S) {
                const float uv = u[y * n + x];
                const float v = uv + fmaf(cf.c1, fmaf(-cf.c0, uv, S), cf.c2 * uv);
                u[y * n + x] = fminf(1.f, fmaxf(-1.f, v));
            });
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        const float x = u[i];
        acc += (double)x;
        if (M.uT) M.uT[(size_t)s * nn + i] = x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < kSqThreads; ++i) tot += red[i];
        const double mean = tot / (double)nn;
        if (M.ubar) M.ubar[s] = mean;
        if (M.ooi) M.ooi[s] = 0.5 * (1.0 + mean);
    }
    __syncthreads();  // the field and red are free for the next item
}

// Persistent CTAs take (model, sample group) items through an atomic ticket counter, heaviest
// model first (the host orders the models), and run each with the fastest form for its lattice.
// SMALL: the launch has register-form items (n = 64, 128), whose 160-odd registers allow one CTA
// per SM; without them the mixed-radix items alone fit two CTAs per SM.
template <bool SMALL>
__global__ void __launch_bounds__(kSqThreads, SMALL ? 1 : 2) spectral_queue_kernel(const __grid_constant__ SqArgs a) {
    extern __shared__ __align__(16) float sq_smem[];
    __shared__ double red[kSqThreads];
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = item;
        __syncthreads();  // every thread has read the ticket before thread 0 takes the next
        if (it >= a.total) break;
        const unsigned long long t0 = a.trace.rec ? trace_clock() : 0ull;
        int k = 0;
        while (k + 1 < a.nm && it >= a.begin[k + 1]) ++k;
        const SqModelDev &M = a.m[k];
        const int local = it - a.begin[k];
        if (SMALL && M.kind == kSqSmall128) {
            if (M.steps_ps)
                small_solve<4, true>(M.u0, M.uT, M.coef, M.khat, M.tw, local, 1, M.steps_ps, M.nsteps, M.ubar, M.ooi,
                                     sq_smem, red);
            else
                small_solve<4, false>(M.u0, M.uT, M.coef, M.khat, M.tw, local, 1, nullptr, M.nsteps, M.ubar, M.ooi,
                                      sq_smem, red);
        } else if (SMALL && M.kind == kSqSmall64) {
            const int s0 = local * SmallCfg<2>::SPC, nloc = min(SmallCfg<2>::SPC, M.ns - s0);
            if (M.steps_ps)
                small_solve<2, true>(M.u0, M.uT, M.coef, M.khat, M.tw, s0, nloc, M.steps_ps, M.nsteps, M.ubar, M.ooi,
                                     sq_smem, red);
            else
                small_solve<2, false>(M.u0, M.uT, M.coef, M.khat, M.tw, s0, nloc, nullptr, M.nsteps, M.ubar, M.ooi,
                                      sq_smem, red);
        } else if (M.plan.n == 88) {
            sq_solve_generic<88>(M, local, sq_smem, red);
        } else {
            sq_solve_generic<0>(M, local, sq_smem, red);
        }
        if (threadIdx.x == 0) trace_put(a.trace, kTraceSpectralQueue, (uint32_t)it, 0, t0);
    }
}

// ----------------------------------------------------------------------------- host side
struct SpectralState {
    int dev = -1;
    size_t cap = 0;
    float2 *khatT = nullptr;  // [513][1024]: K^(ky, kx) / n^2 at [kx][ky], twice (a packed pair)
    float2 *spec = nullptr;   // [cap][1024][528]
    float *bufA = nullptr, *bufB = nullptr;
    float2 *tw = nullptr;     // [32][32]: W_1024^(t k) at [k][t]
    int small_n = 0;          // n = 64 or 128: the resident form's tables
    float *khat_small = nullptr;   // [n/2 + 1][n]: K^(ky, kx) / n^2 at [kx][ky]
    float2 *tw_small = nullptr;    // [E][33]: W_n^(n1 k2) at [n1][k2]
};

void spectral_release(SpectralState *s) {
    if (!s) return;
    cudaFree(s->khatT);
    cudaFree(s->spec);
    cudaFree(s->bufA);
    cudaFree(s->bufB);
    cudaFree(s->tw);
    cudaFree(s->khat_small);
    cudaFree(s->tw_small);
    delete s;
}

bool spectral_supported(const Model &m) {
    const int n = m.d.n;
    return ((n == kN || n == 128 || n == 64) && m.d.bc == MFMC_BC_PERIODIC && m.d.beta2 == 0.0 && 2 * m.R + 1 <= n) ||
           spectral_resident_supported(m);
}

// K^(ky, kx) = sum_dy cos(2 pi ky dy / n) sum_{dx: (dx, dy) in D} w cos(2 pi kx dx / n) (the
// sine terms cancel: the disc and the weights are even in dx and in dy), in FP64 on the host,
// with the weights the FP32 kernels use; divided by n^2 for the two unnormalised inverses.
std::vector<float> spectral_khat(const Model &m, int n) {
    const int R = m.R, half = n / 2 + 1;
    std::vector<double> cs(n);
    for (int i = 0; i < n; ++i) cs[i] = std::cos(2.0 * M_PI * (double)i / (double)n);
    // A[dy][kx] = sum_dx w(dx, dy) cos(2 pi kx dx / n), dy = 0..R
    std::vector<double> A((size_t)(R + 1) * half, 0.0);
    for (int dy = 0; dy <= R; ++dy) {
        const int wd = m.widths[dy];
        for (int kx = 0; kx < half; ++kx) {
            double s = 0.0;
            for (int dx = -wd; dx <= wd; ++dx) {
                const double wt = m.d.kernel == MFMC_KERNEL_CONSTANT ? 1.0 : (double)m.wtab[dx * dx + dy * dy];
                s += wt * cs[(size_t)(((long long)kx * (dx + n)) % n)];
            }
            A[(size_t)dy * half + kx] = s;
        }
    }
    std::vector<float> kh((size_t)half * n);
    const double scale = 1.0 / ((double)n * n);
    for (int ky = 0; ky < n; ++ky)
        for (int kx = 0; kx < half; ++kx) {
            double s = A[kx];  // dy = 0
            for (int dy = 1; dy <= R; ++dy) s += 2.0 * cs[(size_t)((long long)ky * dy % n)] * A[(size_t)dy * half + kx];
            kh[(size_t)kx * n + ky] = (float)(s * scale);
        }
    return kh;
}

// The register transforms' twiddles (c_w32), written once per device before the first
// spectral launch of either form.
static mfmc_status spectral_constants() {
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::vector<bool> consts_set;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)consts_set.size() <= dev) consts_set.resize(dev + 1, false);
    if (!consts_set[dev]) {
        float2 w[kSq];
        for (int k = 0; k < kSq; ++k)
            w[k] = make_float2((float)std::cos(2.0 * M_PI * k / kSq), (float)-std::sin(2.0 * M_PI * k / kSq));
        MFMC_CUDA(cudaMemcpyToSymbol(c_w32, w, sizeof(w)));
        consts_set[dev] = true;
    }
    return MFMC_OK;
}

static mfmc_status spectral_prepare(Model &m, size_t ns) {
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    {
        const mfmc_status cs = spectral_constants();
        if (cs != MFMC_OK) return cs;
    }
    if (!m.d_status) {
        MFMC_CUDA(cudaMalloc((void **)&m.d_status, sizeof(int)));
        MFMC_CUDA(cudaMemset(m.d_status, 0, sizeof(int)));
    }
    if (!m.spectral) m.spectral = new SpectralState();
    SpectralState &s = *m.spectral;
    if (s.dev != dev || !s.khatT) {
        cudaFree(s.khatT);
        cudaFree(s.tw);
        s.khatT = nullptr;
        s.tw = nullptr;
        const std::vector<float> kh = spectral_khat(m, kN);
        std::vector<float2> tw((size_t)kSq * kSq);
        for (int k = 0; k < kSq; ++k)
            for (int t = 0; t < kSq; ++t) {
                const long long e = (long long)t * k % kN;
                tw[(size_t)k * kSq + t] =
                    make_float2((float)std::cos(2.0 * M_PI * e / kN), (float)-std::sin(2.0 * M_PI * e / kN));
            }
        std::vector<float2> kh2(kh.size());
        for (size_t i = 0; i < kh.size(); ++i) kh2[i] = make_float2(kh[i], kh[i]);
        MFMC_CUDA(cudaMalloc((void **)&s.khatT, kh2.size() * sizeof(float2)));
        MFMC_CUDA(cudaMemcpy(s.khatT, kh2.data(), kh2.size() * sizeof(float2), cudaMemcpyHostToDevice));
        MFMC_CUDA(cudaMalloc((void **)&s.tw, tw.size() * sizeof(float2)));
        MFMC_CUDA(cudaMemcpy(s.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
        s.dev = dev;
    }
    if (s.cap < ns) {
        cudaFree(s.spec);
        cudaFree(s.bufA);
        cudaFree(s.bufB);
        s.spec = nullptr;
        s.bufA = s.bufB = nullptr;
        s.cap = 0;
        MFMC_CUDA(cudaMalloc((void **)&s.spec, ns * (size_t)kN * kPitch * sizeof(float2)));
        MFMC_CUDA(cudaMalloc((void **)&s.bufA, ns * (size_t)kN * kN * sizeof(float)));
        MFMC_CUDA(cudaMalloc((void **)&s.bufB, ns * (size_t)kN * kN * sizeof(float)));
        // padding columns 513..527 are transformed by the column pass but never read: defined
        MFMC_CUDA(cudaMemset(s.spec, 0, ns * (size_t)kN * kPitch * sizeof(float2)));
        s.cap = ns;
    }
    return MFMC_OK;
}

// The register form's tables for n = 32 E (once per model and device): K^ / n^2 at [kx][ky] and
// W_n^(n1 k2) at [n1][k2]; the register transforms' constants first.
template <int E>
static mfmc_status small_tables(Model &m, const float **khatT, const float2 **twp) {
    using C = SmallCfg<E>;
    constexpr int N = C::N;
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    {
        const mfmc_status cs = spectral_constants();
        if (cs != MFMC_OK) return cs;
    }
    if (!m.spectral) m.spectral = new SpectralState();
    SpectralState &f = *m.spectral;
    if (f.dev != dev || f.small_n != N || !f.khat_small) {
        cudaFree(f.khat_small);
        cudaFree(f.tw_small);
        f.khat_small = nullptr;
        f.tw_small = nullptr;
        const std::vector<float> kh = spectral_khat(m, N);
        std::vector<float2> tw((size_t)E * 33, make_float2(0.f, 0.f));
        for (int n1 = 0; n1 < E; ++n1)
            for (int k2 = 0; k2 < kSq; ++k2) {
                const long long e = (long long)n1 * k2 % N;
                tw[(size_t)n1 * 33 + k2] =
                    make_float2((float)std::cos(2.0 * M_PI * e / N), (float)-std::sin(2.0 * M_PI * e / N));
            }
        MFMC_CUDA(cudaMalloc((void **)&f.khat_small, kh.size() * sizeof(float)));
        MFMC_CUDA(cudaMemcpy(f.khat_small, kh.data(), kh.size() * sizeof(float), cudaMemcpyHostToDevice));
        MFMC_CUDA(cudaMalloc((void **)&f.tw_small, tw.size() * sizeof(float2)));
        MFMC_CUDA(cudaMemcpy(f.tw_small, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
        f.small_n = N;
        f.dev = dev;
    }
    *khatT = f.khat_small;
    *twp = f.tw_small;
    return MFMC_OK;
}

mfmc_status spectral_small_tables(Model &m, const float **khatT, const float2 **tw) {
    if (m.d.n == 128) return small_tables<4>(m, khatT, tw);
    if (m.d.n == 64) return small_tables<2>(m, khatT, tw);
    return fail(MFMC_EINVAL, "the register-transform form serves n = 64 and 128");
}

size_t spectral_queue_smem(int kind, int n) {
    if (kind == kSqSmall128) return SmallCfg<4>::SMEM;
    if (kind == kSqSmall64) return SmallCfg<2>::SMEM;
    return (size_t)n * n * sizeof(float) + fft_smem_bytes<float>(n, kSqThreads / 32);
}

int spectral_queue_blocks_per_sm(bool small, size_t smem) {
    auto kern = small ? spectral_queue_kernel<true> : spectral_queue_kernel<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kSqThreads, smem);
    (void)cudaGetLastError();  // a failed query must not be reported by a later launch check
    return e == cudaSuccess && per > 0 ? per : 1;
}

mfmc_status launch_spectral_queue(bool small, const SqArgs &a, int grid, size_t smem, cudaStream_t st) {
    auto kern = small ? spectral_queue_kernel<true> : spectral_queue_kernel<false>;
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kSqThreads, smem, st>>>(a);
    MFMC_LAUNCHED("spectral queue launch");
    return MFMC_OK;
}

// The resident form for n = 64 and 128: tables once per model, one launch for the whole solve.
template <int E>
static mfmc_status run_solve_spectral_small(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                                            float *uT, double *ubar, double *ooi, cudaStream_t st) {
    using C = SmallCfg<E>;
    const float *khatT = nullptr;
    const float2 *tw = nullptr;
    const mfmc_status s = small_tables<E>(m, &khatT, &tw);
    if (s != MFMC_OK) return s;
    auto kern = spectral_small_kernel<E>;
    MFMC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    const unsigned grid = (unsigned)((ns + C::SPC - 1) / C::SPC);
    kern<<<grid, C::WARPS * 32, C::SMEM, st>>>(u0, uT, coef, khatT, tw, (int)ns, nsteps, ubar, ooi);
    MFMC_LAUNCHED("spectral launch 4");
    return MFMC_OK;
}

mfmc_status run_solve_spectral(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps, float *uT,
                               double *ubar, double *ooi, cudaStream_t st) {
    if (!spectral_supported(m))
        return fail(MFMC_EINVAL, "the spectral path needs n = 1024 or an even n <= 128 whose odd part factors into 3, "
                                 "5, 7 and 11, a periodic lattice and beta2 = 0");
    {
        int one = 0;
        MFMC_CUDA(cudaDeviceGetAttribute(&one, cudaDevAttrMaxGridDimX, 0));
        if (ns > (size_t)one) return fail(MFMC_EINVAL, "batch too large for the spectral path");
    }
    if (m.d.n == 128) return run_solve_spectral_small<4>(m, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (m.d.n == 64) return run_solve_spectral_small<2>(m, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (m.d.n != kN) return run_solve_spectral_resident(m, coef, u0, ns, nsteps, uT, ubar, ooi, st);
    mfmc_status s = spectral_prepare(m, ns);
    if (s != MFMC_OK) return s;
    SpectralState &f = *m.spectral;
    int dev = 0, sms = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    MFMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t col_smem = ((size_t)kN * kColStride + kSq * kSq) * sizeof(float2);
    const size_t row_smem = ((size_t)kSq * kSq + (size_t)kRowWarps * 2 * kRowBuf) * sizeof(float2);
    MFMC_CUDA(cudaFuncSetAttribute(spectral_column_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem));
    MFMC_CUDA(cudaFuncSetAttribute(spectral_row_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    MFMC_CUDA(cudaFuncSetAttribute(spectral_row_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    MFMC_CUDA(cudaFuncSetAttribute(spectral_row_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    // (a time loop over groups of samples whose spectra stay in L2 measured slower: at 8, 16
    // and 64 samples a launch 7.3, 6.3 and 5.8 us per sample-step)
    const long long pairs = (long long)ns * (kN / 2);
    const unsigned row_grid = (unsigned)std::min<long long>((pairs + kRowWarps - 1) / kRowWarps, (long long)sms);
    const dim3 col_grid(kPitch / kColTile, (unsigned)ns);
    spectral_row_kernel<false, true><<<row_grid, kRowWarps * 32, row_smem, st>>>(f.spec, u0, nullptr, coef, f.tw, pairs,
                                                                                m.d_status);
    MFMC_LAUNCHED("spectral launch 1");
    const float *src = u0;
    for (int k = 1; k <= nsteps; ++k) {
        float *dst = (k == nsteps && uT) ? uT : ((k & 1) ? f.bufA : f.bufB);
        spectral_column_kernel<<<col_grid, kColTile * 32, col_smem, st>>>(f.spec, f.khatT, f.tw);
        MFMC_LAUNCHED("spectral launch 2");
        if (k < nsteps)
            spectral_row_kernel<true, true><<<row_grid, kRowWarps * 32, row_smem, st>>>(f.spec, src, dst, coef, f.tw,
                                                                                       pairs, m.d_status);
        else
            spectral_row_kernel<true, false><<<row_grid, kRowWarps * 32, row_smem, st>>>(f.spec, src, dst, coef, f.tw,
                                                                                        pairs, m.d_status);
        MFMC_LAUNCHED("spectral launch 3");
        src = dst;
    }
    return launch_field_ooi(src, ns, kN, ubar, ooi, st);
}

}  // namespace mfmc
