// The beta2 > 0 step of Eq. (nonl_CH_nm) (MFMC_ALGO_ACTIVE_SET).
//
// Implicit Euler with the convolution explicit: with g = gamma * u^{k-1} + c_F u^{k-1},
//     (u - u^{k-1}) / tau + beta1 w - beta2 Lap_h w = 0,   w in c_gamma u - g + dI(u),
// Lap_h the periodic 5-point Laplacian.  The resolvent of the indicator gives
// u = P_[-1,1]((w + g) / c_gamma), and w solves the strongly monotone equation
//     F(w) = tau (beta1 - beta2 Lap_h) w + P_[-1,1]((w + g) / c_gamma) - u^{k-1} = 0,
// by a semismooth Newton iteration (primal-dual active set): with the inactive set
// I = { |w + g| < c_gamma }, J = tau (beta1 - beta2 Lap_h) + diag(1_I) / c_gamma is symmetric
// positive definite.  The iteration starts from the beta2 = 0 step and stops when the active
// set repeats and max |F| <= 1e-11.
//
// Precision: u, g, w and the residual F are FP64.  Each Newton correction d solves
// J d = -F / max|F| in FP32 to a max-norm residual of 1e-5 (inexact Newton): F is piecewise
// linear in w, so while the active set holds one correction cuts max|F| by about that factor,
// and the FP64 residual of the next iteration sets the accuracy reached.  FP64 arithmetic runs
// at a small fraction of the FP32 rate on GB300, so only the explicit convolution and the
// residual stay in FP64.  The FP32 solve is conjugate gradients preconditioned by one geometric
// multigrid V-cycle (periodic levels, damped Jacobi smoothing, full weighting and bilinear
// prolongation: a symmetric positive definite preconditioner).
//
// The explicit disc sum is FP64 too: a direct sum for small discs, else spectral, which costs
// O(n^2 log n) FP64 operations per field instead of O(n^2 |D|): for n <= 128 by the CTA itself
// (the mixed-radix transforms of smem_fft.cuh, the half spectrum in the shared memory that the
// coarse multigrid levels use during the Newton iteration), for larger n through cuFFT (D2Z, a
// product with the real spectrum of the radial weights, Z2D) between per-step launches.
//
// Newton starts from the previous step's w (the first step from the beta2 = 0 step): the
// solution moves by O(tau) per step, and on the paper's models this start needs about 40 % fewer
// corrections than the beta2 = 0 step, whose residual -tau beta2 Lap_h w is large at interfaces.
//
// One CTA per sample runs every step of its solve (every step of one launch, except with the
// cuFFT sums: one step per launch, the state staying in global scratch between launches); its
// fine-level vectors live in global scratch, the coarse multigrid levels that fit in shared
// memory, and the CTA's reductions use a fixed order.  No CTA waits on another.  Every loop is
// bounded; a Newton iteration that does not converge within its bound sets the status flag (a CG
// solve that reaches its bound hands its iterate to the next Newton iteration).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mfmc_internal.h"
#include "smem_fft.cuh"
#include "trace.cuh"

namespace mfmc {

constexpr int AS_NT = 512;
constexpr float AS_CG_RTOL = 1e-5f;   // max |J d + F| / max |F| that ends a correction
constexpr int AS_VEC64 = 3;           // u, g, w
constexpr int AS_VEC32 = 7;           // d, r, p, q, inactive mask, z, t
constexpr int AS_MAX_LEVELS = 8;
constexpr int AS_NU = 2;              // damped-Jacobi sweeps before and after each coarse correction
constexpr int AS_NU_COARSE = 16;
constexpr float AS_OMEGA = 0.8f;
constexpr int AS_SPECTRAL_MIN_DISC = 100;  // disc points from which the disc sum is spectral

// Multigrid levels of the CG preconditioner: n_0 = n, halved while even and >= 16 (the coarsest
// has >= 8 points per side).  Returns the level count; sizes[l] = n_l.
__host__ __device__ inline int as_levels(int n, int *sizes) {
    int L = 1;
    sizes[0] = n;
    while (L < AS_MAX_LEVELS && sizes[L - 1] % 2 == 0 && sizes[L - 1] >= 16) {
        sizes[L] = sizes[L - 1] / 2;
        ++L;
    }
    return L;
}

// The coarse levels from as_smem_from(n) on live in dynamic shared memory (at most
// AS_SMEM_BUDGET bytes): their passes are short, and each then costs a shared-memory round trip
// and a barrier instead of a global one.  Returns that level and sets *bytes.
constexpr size_t AS_SMEM_BUDGET = 160 * 1024;
__host__ __device__ inline int as_smem_from(int n, size_t *bytes) {
    int sz[AS_MAX_LEVELS];
    const int L = as_levels(n, sz);
    size_t b = 0;
    int l0 = L;
    for (int l = L - 1; l >= 1; --l) {
        const size_t add = (size_t)4 * sz[l] * sz[l] * sizeof(float);
        if (b + add > AS_SMEM_BUDGET) break;
        b += add;
        l0 = l;
    }
    *bytes = b;
    return l0;
}

// Doubles of scratch per sample: the FP64 fine-level vectors, then (two floats per double) the
// FP32 fine-level vectors and, per coarser level that does not live in shared memory, v, f, r
// and m (the levels from as_smem_from(n) on take no global scratch, which keeps a batch's
// working set smaller for L2).
__host__ __device__ inline size_t as_per_sample(int n) {
    int sz[AS_MAX_LEVELS];
    as_levels(n, sz);
    size_t smem_bytes;
    const int l0 = as_smem_from(n, &smem_bytes);
    size_t f = (size_t)AS_VEC32 * n * n;
    for (int l = 1; l < l0; ++l) f += (size_t)4 * sz[l] * sz[l];
    return (size_t)AS_VEC64 * n * n + (f + 1) / 2;
}

struct ActiveSetArgs {
    const float *u0;
    float *uT;
    double *ubar, *ooi;
    const double *eps;   // per sample, or nullptr: eps_nominal
    double eps_nominal;
    double *buf;         // [ns][per]
    size_t per;          // as_per_sample(n)
    int *status;         // set to 1 when an iteration bound is reached
    unsigned long long *iters;  // [2]: Newton and CG iterations, added by every CTA
    const double *wtab;  // Gaussian: FP64 weight / eps^2 by r^2; nullptr: constant kernel
    int widths[kMaxR + 1];
    int n, R, nsteps;
    int newton_max, cg_max;  // iteration bounds: Newton passes per step, CG iterations per correction
    int load;     // read u0 into the FP64 field first
    int g_given;  // the disc sums of u are in g already (cuFFT form): no sum in the kernel
    int warm;     // the launch's first step starts Newton from w in scratch (a step before it ran)
    int own_fft;  // the disc sums by cta_disc_sums (plan, khat, tw) instead of the direct sum
    FftPlan plan;
    const double *khat;  // K^(ky, kx) / n^2 at [ky][n/2 + 1], FP64
    const double2 *tw;   // W_n^j, j < n
    TraceBuf trace;
    int finish;   // write uT, ubar and the OoI after the last step
    size_t s0;
    double ahat, chat, tau, beta1, beta2, cF;
};

// Visit every lattice point (y, x) of an n x n level: warps walk rows, lanes walk columns, so no
// point index is divided and a warp's loads are contiguous.
template <typename Fn>
__device__ __forceinline__ void as_for(int n, Fn f) {
    for (int y = threadIdx.x >> 5; y < n; y += AS_NT / 32)
        for (int x = threadIdx.x & 31; x < n; x += 32) f(y, x, y * n + x);
}

// The same visit, NP points of a thread at a time: v = f(y, x, i) for all NP, then st(i, v)
// for each, so no store stands between the loads of the NP points and they are in flight
// together (a pass over the vectors in global scratch is bound by their latency otherwise).
template <int NP = 4, typename Fn, typename St>
__device__ __forceinline__ void as_map(int n, Fn f, St st) {
    const int J = (n + 31) >> 5, lane = threadIdx.x & 31;
    int y = threadIdx.x >> 5, j = 0;
    while (y < n) {
        int yy[NP], xx[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            yy[q] = y;
            xx[q] = lane + 32 * j;
            if (++j == J) {
                j = 0;
                y += AS_NT / 32;
            }
        }
        decltype(f(0, 0, 0)) v[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (yy[q] < n && xx[q] < n) v[q] = f(yy[q], xx[q], yy[q] * n + xx[q]);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (yy[q] < n && xx[q] < n) st(yy[q] * n + xx[q], v[q]);
    }
}

// Block-wide sum and maximum in a fixed order (warp trees, then the warps in order).
template <typename T>
__device__ T as_block_sum(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // the previous result has been read
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int i = 0; i < AS_NT / 32; ++i) t += red[i];
        red[AS_NT / 32] = t;
    }
    __syncthreads();
    return red[AS_NT / 32];
}

template <typename T>
__device__ T as_block_max(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) {
        const T u = __shfl_down_sync(0xffffffffu, v, o);
        v = v > u ? v : u;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int i = 0; i < AS_NT / 32; ++i) t = t > red[i] ? t : red[i];
        red[AS_NT / 32] = t;
    }
    __syncthreads();
    return red[AS_NT / 32];
}

__device__ __forceinline__ double as_clip(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

// Periodic 5-point Laplacian of v at (y, x), times h^2.
template <typename T>
__device__ __forceinline__ T as_lap_h2(const T *v, int n, int y, int x) {
    const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    return ((v[y * n + xp] + v[y * n + xm]) + (v[yp * n + x] + v[ym * n + x])) - T(4) * v[y * n + x];
}

// The Newton operator on level l (spacing 2^l h, inactive mask m averaged from the fine one), FP32:
// J v = tau beta1 v + (tau beta2 / h_l^2)(4 v - neighbours) + m v / c_gamma.
struct AsLevel {
    float *v, *f, *r;
    const float *m;
    int n;
    float tb2h;  // tau beta2 / h_l^2
};

__device__ __forceinline__ float as_apply(const AsLevel &L, const float *v, int y, int x, int i, float tb1,
                                          float icg) {
    return tb1 * v[i] - L.tb2h * as_lap_h2(v, L.n, y, x) + L.m[i] * icg * v[i];
}

// One damped-Jacobi sweep on level L: dst = src + omega D^-1 (f - J src), or dst = omega D^-1 f
// when src is nullptr (a sweep from zero).  dst != src.  Returns the thread's partial sum of
// f * dst.
__device__ __noinline__ float as_sweep(const AsLevel &L, const float *src, float *dst, float tb1, float icg) {
    const float dconst = tb1 + 4.0f * L.tb2h;
    float acc = 0.0f;
    auto store = [&](int i, float2 v) {
        dst[i] = v.x;
        acc += v.y;
    };
    if (!src) {
        as_map(L.n, [&](int, int, int i) {
            const float f = L.f[i], v = AS_OMEGA * f / (dconst + L.m[i] * icg);
            return make_float2(v, f * v);
        }, store);
    } else {
        as_map(L.n, [&](int y, int x, int i) {
            const float f = L.f[i], v = src[i] + AS_OMEGA * (f - as_apply(L, src, y, x, i, tb1, icg)) /
                                                     (dconst + L.m[i] * icg);
            return make_float2(v, f * v);
        }, store);
    }
    __syncthreads();
    return acc;
}

// One V-cycle z = B r (levels[0].f = r in, levels[0].v = z out; symmetric: damped Jacobi before
// and after each coarse correction, full-weighting restriction = prolongation transpose / 4).
// Each visit of a level makes an even number of sweeps alternating between v and r, the first
// from zero, so z ends in v.  Returns the thread's partial sum of r * z.
static_assert(AS_NU == 2 && AS_NU_COARSE % 2 == 0, "the sweeps alternate between two buffers");
__device__ __noinline__ float as_vcycle(const AsLevel *lv, int nl, float tb1, float icg) {
    float dot = 0.0f;
    for (int l = 0; l < nl; ++l) {
        const AsLevel &L = lv[l];
        if (l == nl - 1) {
            as_sweep(L, nullptr, L.r, tb1, icg);
            for (int k = 2; k <= AS_NU_COARSE; ++k) {
                const float d = (k & 1) ? as_sweep(L, L.v, L.r, tb1, icg) : as_sweep(L, L.r, L.v, tb1, icg);
                if (l == 0 && k == AS_NU_COARSE) dot = d;
            }
            break;
        }
        as_sweep(L, nullptr, L.r, tb1, icg);
        as_sweep(L, L.r, L.v, tb1, icg);
        as_map(L.n, [&](int y, int x, int i) { return L.f[i] - as_apply(L, L.v, y, x, i, tb1, icg); },
               [&](int i, float v) { L.r[i] = v; });
        __syncthreads();
        const AsLevel &C = lv[l + 1];
        const int n = L.n;
        as_map(C.n, [&](int Y, int X, int) {  // full weighting at (2Y, 2X)
            const int y = 2 * Y, x = 2 * X;
            const int ym = y == 0 ? n - 1 : y - 1, yp = y + 1, xm = x == 0 ? n - 1 : x - 1, xp = x + 1;
            const float c = L.r[y * n + x];
            const float e = (L.r[y * n + xm] + L.r[y * n + xp]) + (L.r[ym * n + x] + L.r[yp * n + x]);
            const float k = (L.r[ym * n + xm] + L.r[ym * n + xp]) + (L.r[yp * n + xm] + L.r[yp * n + xp]);
            return (4.0f * c + 2.0f * e + k) * 0.0625f;
        }, [&](int i, float v) { C.f[i] = v; });
        __syncthreads();
    }
    for (int l = nl - 2; l >= 0; --l) {
        const AsLevel &L = lv[l], &C = lv[l + 1];
        const int nc = C.n;
        as_map(L.n, [&](int y, int x, int i) {  // bilinear prolongation (periodic)
            const int Y = y >> 1, X = x >> 1;
            const int Y1 = (y & 1) ? (Y + 1 == nc ? 0 : Y + 1) : Y, X1 = (x & 1) ? (X + 1 == nc ? 0 : X + 1) : X;
            return L.v[i] + 0.25f * ((C.v[Y * nc + X] + C.v[Y * nc + X1]) + (C.v[Y1 * nc + X] + C.v[Y1 * nc + X1]));
        }, [&](int i, float v) { L.v[i] = v; });
        __syncthreads();
        as_sweep(L, L.v, L.r, tb1, icg);
        const float d = as_sweep(L, L.r, L.v, tb1, icg);
        if (l == 0) dot = d;
    }
    return dot;
}

__global__ void __launch_bounds__(AS_NT) active_set_kernel(ActiveSetArgs a) {
    __shared__ double red64[AS_NT / 32 + 1];
    __shared__ float red32[AS_NT / 32 + 1];
    __shared__ int widths[kMaxR + 1];
    const size_t smp = a.s0 + blockIdx.x;
    const unsigned long long t_start = a.trace.rec ? trace_clock() : 0ull;
    const int n = a.n, R = a.R;
    const int nn = n * n;
    double *U = a.buf + smp * a.per;
    double *G = U + nn, *W = G + nn;
    float *D = reinterpret_cast<float *>(W + nn);
    float *Rr = D + nn, *Pp = Rr + nn, *Q = Pp + nn, *M = Q + nn, *Z = M + nn, *T = Z + nn;
    // multigrid levels of the preconditioner
    int sizes[AS_MAX_LEVELS];
    const int nl = as_levels(n, sizes);
    AsLevel lv[AS_MAX_LEVELS];
    extern __shared__ __align__(16) float as_smem[];
    {
        size_t smem_bytes;
        const int l0 = as_smem_from(n, &smem_bytes);
        float *q = T + nn, *qs = as_smem;  // global levels 1 .. l0 - 1, shared levels l0 ..
        for (int l = 0; l < nl; ++l) {
            const float tb2h_l = (float)(a.tau * a.beta2 * (double)sizes[l] * (double)sizes[l]);
            if (l == 0) {
                lv[0] = AsLevel{Z, Rr, T, M, n, tb2h_l};
            } else {
                const size_t ml = (size_t)sizes[l] * sizes[l];
                float *b = l >= l0 ? qs : q;
                lv[l] = AsLevel{b, b + ml, b + 2 * ml, b + 3 * ml, sizes[l], tb2h_l};
                (l >= l0 ? qs : q) += 4 * ml;
            }
        }
    }
    if (threadIdx.x <= R) widths[threadIdx.x] = a.widths[threadIdx.x];
    const double eps = a.eps ? a.eps[smp] : a.eps_nominal;
    const double e2a = eps * eps * a.ahat;              // h^2 gamma = e2a * what
    const double cg = e2a * a.chat;                     // c_gamma
    const double tb1 = a.tau * a.beta1, tb2h = a.tau * a.beta2 * (double)n * (double)n;  // tau beta2 / h^2
    const float tb1f = (float)tb1, tb2hf = lv[0].tb2h, icgf = (float)(1.0 / cg);
    if (a.load) {
        as_for(n, [&](int, int, int i) { U[i] = (double)a.u0[smp * (size_t)nn + i]; });
        __syncthreads();
    }
    bool failed = false;
    unsigned long long n_newton = 0, n_cg = 0;
    for (int step = 1; step <= a.nsteps && !failed; ++step) {
        // explicit part g = gamma * u + c_F u (direct sum over the disc, FP64; R < n, so one
        // wrap of each index suffices)
        if (a.g_given) as_for(n, [&](int, int, int i) { G[i] = e2a * G[i] + a.cF * U[i]; });
        else if (a.own_fft) {  // (the coarse levels in shared memory hold nothing between steps)
            auto ld = [&](int y, int x) { return U[y * n + x]; };
            auto put = [&](int y, int x, double S) { G[y * n + x] = e2a * S + a.cF * U[y * n + x]; };
            switch (n) {  // the paper's meshes on compile-time plans
                case 64: cta_disc_sums<64, double>(a.plan, as_smem, a.khat, a.tw, ld, put); break;
                case 88: cta_disc_sums<88, double>(a.plan, as_smem, a.khat, a.tw, ld, put); break;
                case 128: cta_disc_sums<128, double>(a.plan, as_smem, a.khat, a.tw, ld, put); break;
                default: cta_disc_sums<0, double>(a.plan, as_smem, a.khat, a.tw, ld, put); break;
            }
        } else as_for(n, [&](int y, int x, int i) {
            double S = 0.0;
            for (int dy = -R; dy <= R; ++dy) {
                const int ady = dy < 0 ? -dy : dy, w = widths[ady];
                int yy = y + dy;
                yy += yy < 0 ? n : 0;
                yy -= yy >= n ? n : 0;
                const double *row = U + (size_t)yy * n;
                int xx = x - w;
                xx += xx < 0 ? n : 0;
                if (a.wtab) {
                    const double *wr = a.wtab + ady * ady;
                    for (int dx = -w; dx <= w; ++dx) {
                        S += wr[dx * dx] * row[xx];
                        xx = xx == n - 1 ? 0 : xx + 1;
                    }
                } else {
                    for (int dx = -w; dx <= w; ++dx) {
                        S += row[xx];
                        xx = xx == n - 1 ? 0 : xx + 1;
                    }
                }
            }
            G[i] = e2a * S + a.cF * U[i];
        });
        __syncthreads();
        // start: w of the previous step, or at the solve's first step the beta2 = 0 step
        // w = c_gamma u0 - g
        if (step == 1 && !a.warm) {
            as_for(n, [&](int, int, int i) {
                const double u0 = as_clip((U[i] + tb1 * G[i]) / (1.0 + tb1 * cg));
                W[i] = cg * u0 - G[i];
            });
            __syncthreads();
        }
        for (int it = 1;; ++it) {
            ++n_newton;
            // FP64 residual F(w), the inactive set, and the right-hand side r = -F of J d = -F
            double fmax = 0.0, changed = 0.0;
            as_for(n, [&](int y, int x, int i) {
                const double xv = (W[i] + G[i]) / cg;
                const float inact = fabs(xv) < 1.0 ? 1.0f : 0.0f;
                const double F = (tb1 * W[i] - tb2h * as_lap_h2(W, n, y, x)) + as_clip(xv) - U[i];
                if (M[i] != inact) changed = 1.0;
                M[i] = inact;
                Rr[i] = (float)(-F);
                D[i] = 0.0f;
                fmax = fmax > fabs(F) ? fmax : fabs(F);
            });
            fmax = as_block_max(fmax, red64);
            changed = as_block_max(changed, red64);
            if (it > 1 && changed == 0.0 && fmax <= 1e-11) break;
            if (it > a.newton_max) {
                failed = true;
                break;
            }
            if (fmax == 0.0) continue;  // F = 0 with a new active set: the next pass confirms it
            // scale to max |r| = 1, and the inactive mask on the coarse levels (2 x 2 averages)
            const float sc = (float)(1.0 / fmax);
            as_for(n, [&](int, int, int i) { Rr[i] *= sc; });
            for (int l = 1; l < nl; ++l) {
                const int nf = sizes[l - 1];
                float *mc = const_cast<float *>(lv[l].m);
                const float *mf = lv[l - 1].m;
                as_for(sizes[l], [&](int Y, int X, int i) {
                    mc[i] = 0.25f * ((mf[2 * Y * nf + 2 * X] + mf[2 * Y * nf + 2 * X + 1]) +
                                     (mf[(2 * Y + 1) * nf + 2 * X] + mf[(2 * Y + 1) * nf + 2 * X + 1]));
                });
                __syncthreads();
            }
            __syncthreads();
            // FP32 CG on J d = r preconditioned by one multigrid V-cycle, d = 0 at the start.  q = J p
            // follows the recurrence q = J z + beta q, so one stencil pass (on z) serves each
            // iteration, and r . z comes out of the V-cycle's last sweep.
            float rz = as_block_sum(as_vcycle(lv, nl, tb1f, icgf), red32);  // Z = B Rr
            float beta = 0.0f;
            for (int k = 1;; ++k) {
                const bool first = k == 1;
                float pq = 0.0f;
                as_map(n, [&](int y, int x, int i) {
                    const float z = Z[i];
                    const float jz = (tb1f * z - tb2hf * as_lap_h2(Z, n, y, x)) + M[i] * icgf * z;
                    return first ? make_float2(z, jz) : make_float2(z + beta * Pp[i], jz + beta * Q[i]);
                }, [&](int i, float2 v) {
                    Pp[i] = v.x;
                    Q[i] = v.y;
                    pq += v.x * v.y;
                });
                pq = as_block_sum(pq, red32);
                const float alpha = pq > 0.0f ? rz / pq : 0.0f;
                float rmax = 0.0f;
                as_map(n, [&](int, int, int i) { return make_float2(D[i] + alpha * Pp[i], Rr[i] - alpha * Q[i]); },
                       [&](int i, float2 v) {
                           D[i] = v.x;
                           Rr[i] = v.y;
                           rmax = rmax > fabsf(v.y) ? rmax : fabsf(v.y);
                       });
                rmax = as_block_max(rmax, red32);
                if (rmax <= AS_CG_RTOL || !(pq > 0.0f) || !(rz > 0.0f) || k >= a.cg_max) {
                    n_cg += k;
                    break;
                }
                const float rz2 = as_block_sum(as_vcycle(lv, nl, tb1f, icgf), red32);  // Z = B Rr
                beta = rz2 / rz;
                rz = rz2;
            }
            as_for(n, [&](int, int, int i) { W[i] += fmax * (double)D[i]; });
            __syncthreads();
        }
        if (failed) break;
        as_for(n, [&](int, int, int i) { U[i] = as_clip((W[i] + G[i]) / cg); });
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&a.iters[0], n_newton);
        atomicAdd(&a.iters[1], n_cg);
        trace_put(a.trace, kTraceActiveSet, (uint32_t)smp, (uint32_t)a.nsteps, t_start);
    }
    if (failed) {
        if (threadIdx.x == 0) atomicExch(a.status, 1);
        return;
    }
    if (!a.finish) return;
    double s = 0.0;
    as_for(n, [&](int, int, int i) {
        s += U[i];
        if (a.uT) a.uT[smp * (size_t)nn + i] = (float)U[i];
    });
    s = as_block_sum(s, red64);
    if (threadIdx.x == 0) {
        const double mean = s / (double)nn;
        if (a.ubar) a.ubar[smp] = mean;
        if (a.ooi) a.ooi[smp] = 0.5 * (1.0 + mean);
    }
}

mfmc_status run_solve_active_set(Model &m, const double *eps_dev, const float *u0, size_t ns, int nsteps,
                                 float *uT, double *ubar, double *ooi, cudaStream_t st) {
    if (!(m.d.beta2 > 0.0)) return fail(MFMC_EINVAL, "the active-set solver is for beta2 > 0");
    if (ns == 0) return MFMC_OK;
    const size_t per = as_per_sample(m.d.n);
    mfmc_status s = grow_buffer(&m.as_buf, &m.as_cap, ns * per);
    if (s != MFMC_OK) return s;
    if (!m.d_status) {
        MFMC_CUDA(cudaMalloc((void **)&m.d_status, sizeof(int)));
        MFMC_CUDA(cudaMemset(m.d_status, 0, sizeof(int)));
    }
    if (m.d.kernel == MFMC_KERNEL_GAUSSIAN && !m.d_wtab64) {
        MFMC_CUDA(cudaMalloc((void **)&m.d_wtab64, m.wtab64.size() * sizeof(double)));
        MFMC_CUDA(cudaMemcpy(m.d_wtab64, m.wtab64.data(), m.wtab64.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (!m.d_as_iters) MFMC_CUDA(cudaMalloc((void **)&m.d_as_iters, 2 * sizeof(unsigned long long)));
    MFMC_CUDA(cudaMemsetAsync(m.d_as_iters, 0, 2 * sizeof(unsigned long long), st));
    // the inactive-set vector starts at an impossible value, so no step sees a stale set
    MFMC_CUDA(cudaMemsetAsync(m.as_buf, 0xff, ns * per * sizeof(double), st));
    ActiveSetArgs a;
    a.u0 = u0;
    a.uT = uT;
    a.ubar = ubar;
    a.ooi = ooi;
    a.eps = eps_dev;
    a.eps_nominal = m.d.eps;
    a.buf = m.as_buf;
    a.per = per;
    a.status = m.d_status;
    a.iters = m.d_as_iters;
    a.wtab = m.d.kernel == MFMC_KERNEL_GAUSSIAN ? m.d_wtab64 : nullptr;
    for (int d = 0; d <= kMaxR; ++d) a.widths[d] = d <= m.R ? m.widths[d] : 0;
    a.n = m.d.n;
    a.R = m.R;
    a.newton_max = m.as_newton_max;
    a.cg_max = m.as_cg_max;
    a.ahat = m.ahat;
    a.chat = m.chat64;
    a.tau = m.d.tau;
    a.beta1 = m.d.beta1;
    a.beta2 = m.d.beta2;
    a.cF = m.d.c_F;
    // the disc sums: direct for small discs; else spectral, by the CTA's own transforms when the
    // half spectrum fits in shared memory beside nothing else, else through cuFFT
    size_t smem = 0;
    as_smem_from(m.d.n, &smem);
    const bool spectral = m.disc >= AS_SPECTRAL_MIN_DISC;
    FftPlan plan;
    const bool own = spectral && m.d.n <= kFftMaxN && m.d.n % 2 == 0 && fft_plan(m.d.n, &plan);
    a.own_fft = own ? 1 : 0;
    a.plan = plan;
    a.khat = nullptr;
    a.tw = nullptr;
    a.warm = 0;
    a.trace = trace_buf();
    if (own) {
        const int n = m.d.n;
        if (!m.d_khat64) {
            const std::vector<double> K = khat64_host(m, n);
            std::vector<double2> tw(n);
            for (int j = 0; j < n; ++j)
                tw[j] = make_double2(std::cos(2.0 * M_PI * j / n), -std::sin(2.0 * M_PI * j / n));
            MFMC_CUDA(cudaMalloc((void **)&m.d_khat64, K.size() * sizeof(double)));
            MFMC_CUDA(cudaMemcpy(m.d_khat64, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice));
            MFMC_CUDA(cudaMalloc((void **)&m.d_tw64, tw.size() * sizeof(double2)));
            MFMC_CUDA(cudaMemcpy(m.d_tw64, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
        }
        a.khat = m.d_khat64;
        a.tw = m.d_tw64;
        smem = std::max(smem, fft_smem_bytes<double>(n, AS_NT / 32));
    }
    MFMC_CUDA(cudaFuncSetAttribute(active_set_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    auto launch = [&](int load, int steps, int g_given, int finish) -> mfmc_status {
        a.load = load;
        a.nsteps = steps;
        a.g_given = g_given;
        a.finish = finish;
        for (size_t o = 0; o < ns; o += 65535) {
            a.s0 = o;
            active_set_kernel<<<(unsigned)std::min<size_t>(65535, ns - o), AS_NT, smem, st>>>(a);
            MFMC_LAUNCHED("active_set launch 1");
        }
        return MFMC_OK;
    };
    if (!spectral || own || !fft64_available()) return launch(1, nsteps, 0, 1);
    // cuFFT disc sums: g of sample s (at u + n^2 in its block) from u, between one-step launches
    const size_t nn = (size_t)m.d.n * m.d.n;
    s = launch(1, 0, 0, nsteps == 0);
    for (int k = 1; k <= nsteps && s == MFMC_OK; ++k) {
        s = fft64_disc_sums(m, m.as_buf, per, m.as_buf + nn, per, ns, st);
        a.warm = k > 1;
        if (s == MFMC_OK) s = launch(0, 1, 1, k == nsteps);
    }
    return s;
}

}  // namespace mfmc
