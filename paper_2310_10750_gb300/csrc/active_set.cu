// The beta2 > 0 step of Eq. (nonl_CH_nm) (MFMC_ALGO_ACTIVE_SET).
//
// Implicit Euler with the convolution explicit: with g = gamma * u^{k-1} + c_F u^{k-1},
//     (u - u^{k-1}) / tau + beta1 w - beta2 Lap_h w = 0,   w in c_gamma u - g + dI(u),
// Lap_h the periodic 5-point Laplacian.  The resolvent of the indicator gives
// u = P_[-1,1]((w + g) / c_gamma), and w solves the strongly monotone equation
//     F(w) = tau (beta1 - beta2 Lap_h) w + P_[-1,1]((w + g) / c_gamma) - u^{k-1} = 0,
// by a semismooth Newton iteration (primal-dual active set): with the inactive set
// I = { |w + g| < c_gamma }, J = tau (beta1 - beta2 Lap_h) + diag(1_I) / c_gamma is symmetric
// positive definite and each Newton system is solved by conjugate gradients preconditioned by
// one geometric multigrid V-cycle (periodic levels, damped Jacobi smoothing, full weighting and
// bilinear prolongation: a symmetric positive definite preconditioner).  The iteration starts from the beta2 = 0 step and stops when the active set
// repeats and max |F| is at rounding level.
//
// One CTA per sample runs every step of its solve; its vectors live in global scratch (FP64)
// and the CTA's reductions use a fixed order.  No CTA waits on another.  Every loop is bounded;
// a Newton or CG iteration that does not converge within its bound sets the status flag.
#include <cuda_runtime.h>

#include <algorithm>

#include "mfmc_internal.h"

namespace mfmc {

constexpr int AS_NT = 512;
constexpr int AS_MAX_NEWTON = 60;
constexpr int AS_MAX_CG = 40000;
constexpr int AS_VECS = 10;  // u, g, w, d, r, p, q, inactive mask, z, t
constexpr int AS_MAX_LEVELS = 8;
constexpr int AS_NU = 2;        // damped-Jacobi sweeps before and after each coarse correction
constexpr int AS_NU_COARSE = 16;
constexpr double AS_OMEGA = 0.8;

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

// Doubles of scratch per sample: the fine-level vectors and, per coarser level, v, f, r and m.
__host__ __device__ inline size_t as_per_sample(int n) {
    int sz[AS_MAX_LEVELS];
    const int L = as_levels(n, sz);
    size_t t = (size_t)AS_VECS * n * n;
    for (int l = 1; l < L; ++l) t += (size_t)4 * sz[l] * sz[l];
    return t;
}

struct ActiveSetArgs {
    const float *u0;
    float *uT;
    double *ubar, *ooi;
    const double *eps;   // per sample, or nullptr: eps_nominal
    double eps_nominal;
    double *buf;         // [ns][as_per_sample(n)]
    int *status;         // set to 1 when an iteration bound is reached
    const double *wtab;  // Gaussian: FP64 weight / eps^2 by r^2; nullptr: constant kernel
    int widths[kMaxR + 1];
    int n, R, nsteps;
    size_t s0;
    double ahat, chat, tau, beta1, beta2, cF;
};

// Block-wide sum and maximum in a fixed order (warp trees, then the warps in order).
__device__ double as_block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // the previous result has been read
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < AS_NT / 32; ++i) t += red[i];
        red[AS_NT / 32] = t;
    }
    __syncthreads();
    return red[AS_NT / 32];
}

__device__ double as_block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < AS_NT / 32; ++i) t = fmax(t, red[i]);
        red[AS_NT / 32] = t;
    }
    __syncthreads();
    return red[AS_NT / 32];
}

__device__ __forceinline__ double as_clip(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

// Periodic 5-point Laplacian of v at (y, x), times h^2.
__device__ __forceinline__ double as_lap_h2(const double *v, int n, int y, int x) {
    const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    return ((v[y * n + xp] + v[y * n + xm]) + (v[yp * n + x] + v[ym * n + x])) - 4.0 * v[y * n + x];
}

// The Newton operator on level l (spacing 2^l h, inactive mask m averaged from the fine one):
// J v = tau beta1 v + (tau beta2 / h_l^2)(4 v - neighbours) + m v / c_gamma.
struct AsLevel {
    double *v, *f, *r;
    const double *m;
    int n;
    double tb2h;  // tau beta2 / h_l^2
};

__device__ __forceinline__ double as_apply(const AsLevel &L, const double *v, int i, double tb1, double cg) {
    const int n = L.n, y = i / n, x = i - y * n;
    return tb1 * v[i] - L.tb2h * as_lap_h2(v, n, y, x) + L.m[i] * v[i] / cg;
}

__device__ __forceinline__ double as_diag(const AsLevel &L, int i, double tb1, double cg) {
    return tb1 + 4.0 * L.tb2h + L.m[i] / cg;
}

// nu damped-Jacobi sweeps on level L (v <- v + omega D^-1 (f - J v)), r as the temporary
__device__ void as_smooth(const AsLevel &L, int nu, double tb1, double cg) {
    const int nn = L.n * L.n;
    for (int k = 0; k < nu; ++k) {
        for (int i = threadIdx.x; i < nn; i += AS_NT) L.r[i] = L.f[i] - as_apply(L, L.v, i, tb1, cg);
        __syncthreads();
        for (int i = threadIdx.x; i < nn; i += AS_NT) L.v[i] += AS_OMEGA * L.r[i] / as_diag(L, i, tb1, cg);
        __syncthreads();
    }
}

// One V-cycle z = B r (symmetric: damped Jacobi before and after each correction, full-weighting
// restriction = prolongation transpose / 4), levels[0].f = r and levels[0].v = z.
__device__ void as_vcycle(const AsLevel *lv, int nl, double tb1, double cg) {
    for (int l = 0; l < nl; ++l) {
        const AsLevel &L = lv[l];
        const int nn = L.n * L.n;
        for (int i = threadIdx.x; i < nn; i += AS_NT) L.v[i] = 0.0;
        __syncthreads();
        if (l == nl - 1) {
            as_smooth(L, AS_NU_COARSE, tb1, cg);
            break;
        }
        as_smooth(L, AS_NU, tb1, cg);
        for (int i = threadIdx.x; i < nn; i += AS_NT) L.r[i] = L.f[i] - as_apply(L, L.v, i, tb1, cg);
        __syncthreads();
        const AsLevel &C = lv[l + 1];
        const int nc = C.n, n = L.n;
        for (int i = threadIdx.x; i < nc * nc; i += AS_NT) {  // full weighting at (2Y, 2X)
            const int Y = i / nc, X = i - Y * nc, y = 2 * Y, x = 2 * X;
            const int ym = y == 0 ? n - 1 : y - 1, yp = y + 1, xm = x == 0 ? n - 1 : x - 1, xp = x + 1;
            const double c = L.r[y * n + x];
            const double e = (L.r[y * n + xm] + L.r[y * n + xp]) + (L.r[ym * n + x] + L.r[yp * n + x]);
            const double k = (L.r[ym * n + xm] + L.r[ym * n + xp]) + (L.r[yp * n + xm] + L.r[yp * n + xp]);
            C.f[i] = (4.0 * c + 2.0 * e + k) / 16.0;
        }
        __syncthreads();
    }
    for (int l = nl - 2; l >= 0; --l) {
        const AsLevel &L = lv[l], &C = lv[l + 1];
        const int n = L.n, nc = C.n, nn = n * n;
        for (int i = threadIdx.x; i < nn; i += AS_NT) {  // bilinear prolongation (periodic)
            const int y = i / n, x = i - y * n, Y = y >> 1, X = x >> 1;
            const int Y1 = (y & 1) ? (Y + 1 == nc ? 0 : Y + 1) : Y, X1 = (x & 1) ? (X + 1 == nc ? 0 : X + 1) : X;
            const double v = 0.25 * ((C.v[Y * nc + X] + C.v[Y * nc + X1]) + (C.v[Y1 * nc + X] + C.v[Y1 * nc + X1]));
            L.v[i] += v;
        }
        __syncthreads();
        as_smooth(L, AS_NU, tb1, cg);
    }
}

__global__ void __launch_bounds__(AS_NT) active_set_kernel(ActiveSetArgs a) {
    __shared__ double red[AS_NT / 32 + 1];
    __shared__ int widths[kMaxR + 1];
    const size_t smp = a.s0 + blockIdx.x;
    const int n = a.n, R = a.R;
    const int nn = n * n;
    double *U = a.buf + smp * as_per_sample(n);
    double *G = U + nn, *W = G + nn, *D = W + nn, *Rr = D + nn, *Pp = Rr + nn, *Q = Pp + nn, *M = Q + nn;
    double *Z = M + nn, *T = Z + nn;
    // multigrid levels of the preconditioner
    int sizes[AS_MAX_LEVELS];
    const int nl = as_levels(n, sizes);
    AsLevel lv[AS_MAX_LEVELS];
    {
        double *q = T + nn;
        for (int l = 0; l < nl; ++l) {
            const double tb2h_l = a.tau * a.beta2 * (double)sizes[l] * (double)sizes[l];
            if (l == 0) {
                lv[0] = AsLevel{Z, Rr, T, M, n, tb2h_l};
            } else {
                const size_t ml = (size_t)sizes[l] * sizes[l];
                lv[l] = AsLevel{q, q + ml, q + 2 * ml, q + 3 * ml, sizes[l], tb2h_l};
                q += 4 * ml;
            }
        }
    }
    if (threadIdx.x <= R) widths[threadIdx.x] = a.widths[threadIdx.x];
    const double eps = a.eps ? a.eps[smp] : a.eps_nominal;
    const double e2a = eps * eps * a.ahat;              // h^2 gamma = e2a * what
    const double cg = e2a * a.chat;                     // c_gamma
    const double tb1 = a.tau * a.beta1, tb2h = a.tau * a.beta2 * (double)n * (double)n;  // tau beta2 / h^2
    for (int i = threadIdx.x; i < nn; i += AS_NT) U[i] = (double)a.u0[smp * (size_t)nn + i];
    __syncthreads();
    bool failed = false;
    for (int step = 1; step <= a.nsteps && !failed; ++step) {
        // explicit part g = gamma * u + c_F u (direct sum over the disc, FP64)
        for (int i = threadIdx.x; i < nn; i += AS_NT) {
            const int y = i / n, x = i - y * n;
            double S = 0.0;
            for (int dy = -R; dy <= R; ++dy) {
                const int w = widths[dy < 0 ? -dy : dy];
                const double *row = U + (size_t)((y + dy + n) % n) * n;
                for (int dx = -w; dx <= w; ++dx) {
                    const double v = row[(x + dx + n) % n];
                    S += a.wtab ? a.wtab[dx * dx + dy * dy] * v : v;
                }
            }
            G[i] = e2a * S + a.cF * U[i];
        }
        __syncthreads();
        // start: the beta2 = 0 step, w = c_gamma u0 - g
        for (int i = threadIdx.x; i < nn; i += AS_NT) {
            const double u0 = as_clip((U[i] + tb1 * G[i]) / (1.0 + tb1 * cg));
            W[i] = cg * u0 - G[i];
        }
        __syncthreads();
        for (int it = 1;; ++it) {
            // residual F(w), the inactive set, and the right-hand side r = -F of J d = -F
            double fmax = 0.0, changed = 0.0;
            for (int i = threadIdx.x; i < nn; i += AS_NT) {
                const int y = i / n, x = i - y * n;
                const double xv = (W[i] + G[i]) / cg;
                const double inact = fabs(xv) < 1.0 ? 1.0 : 0.0;
                const double F = (tb1 * W[i] - tb2h * as_lap_h2(W, n, y, x)) + as_clip(xv) - U[i];
                if (M[i] != inact) changed = 1.0;
                M[i] = inact;
                Rr[i] = -F;
                D[i] = 0.0;
                fmax = fmax > fabs(F) ? fmax : fabs(F);
            }
            fmax = as_block_max(fmax, red);
            changed = as_block_max(changed, red);
            if (it > 1 && changed == 0.0 && fmax <= 1e-11) break;
            if (it > AS_MAX_NEWTON) {
                failed = true;
                break;
            }
            // the inactive mask on the coarse levels (2 x 2 averages)
            for (int l = 1; l < nl; ++l) {
                const int nc = sizes[l], nf = sizes[l - 1];
                double *mc = const_cast<double *>(lv[l].m);
                const double *mf = lv[l - 1].m;
                for (int i = threadIdx.x; i < nc * nc; i += AS_NT) {
                    const int Y = i / nc, X = i - Y * nc;
                    mc[i] = 0.25 * ((mf[2 * Y * nf + 2 * X] + mf[2 * Y * nf + 2 * X + 1]) +
                                    (mf[(2 * Y + 1) * nf + 2 * X] + mf[(2 * Y + 1) * nf + 2 * X + 1]));
                }
                __syncthreads();
            }
            // CG on J d = r preconditioned by one multigrid V-cycle, d = 0 at the start
            as_vcycle(lv, nl, tb1, cg);  // Z = B Rr
            double rz = 0.0;
            for (int i = threadIdx.x; i < nn; i += AS_NT) {
                Pp[i] = Z[i];
                rz += Rr[i] * Z[i];
            }
            rz = as_block_sum(rz, red);
            const double rtol = fmax * 1e-6 > 1e-13 ? fmax * 1e-6 : 1e-13;
            for (int k = 1;; ++k) {
                double pq = 0.0;
                for (int i = threadIdx.x; i < nn; i += AS_NT) {
                    const int y = i / n, x = i - y * n;
                    const double q = (tb1 * Pp[i] - tb2h * as_lap_h2(Pp, n, y, x)) + M[i] * Pp[i] / cg;
                    Q[i] = q;
                    pq += Pp[i] * q;
                }
                pq = as_block_sum(pq, red);
                const double alpha = pq > 0.0 ? rz / pq : 0.0;
                double rmax = 0.0;
                for (int i = threadIdx.x; i < nn; i += AS_NT) {
                    D[i] += alpha * Pp[i];
                    Rr[i] -= alpha * Q[i];
                    rmax = rmax > fabs(Rr[i]) ? rmax : fabs(Rr[i]);
                }
                rmax = as_block_max(rmax, red);
                if (rmax <= rtol || pq <= 0.0) break;
                if (k >= AS_MAX_CG) {
                    failed = true;
                    break;
                }
                __syncthreads();
                as_vcycle(lv, nl, tb1, cg);  // Z = B Rr
                double rz2 = 0.0;
                for (int i = threadIdx.x; i < nn; i += AS_NT) rz2 += Rr[i] * Z[i];
                rz2 = as_block_sum(rz2, red);
                const double beta = rz2 / rz;
                rz = rz2;
                for (int i = threadIdx.x; i < nn; i += AS_NT) Pp[i] = Z[i] + beta * Pp[i];
                __syncthreads();
            }
            if (failed) break;
            for (int i = threadIdx.x; i < nn; i += AS_NT) W[i] += D[i];
            __syncthreads();
        }
        if (failed) break;
        for (int i = threadIdx.x; i < nn; i += AS_NT) U[i] = as_clip((W[i] + G[i]) / cg);
        __syncthreads();
    }
    if (failed) {
        if (threadIdx.x == 0) atomicExch(a.status, 1);
        return;
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < nn; i += AS_NT) {
        s += U[i];
        if (a.uT) a.uT[smp * (size_t)nn + i] = (float)U[i];
    }
    s = as_block_sum(s, red);
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
    a.status = m.d_status;
    a.wtab = m.d.kernel == MFMC_KERNEL_GAUSSIAN ? m.d_wtab64 : nullptr;
    for (int d = 0; d <= kMaxR; ++d) a.widths[d] = d <= m.R ? m.widths[d] : 0;
    a.n = m.d.n;
    a.R = m.R;
    a.nsteps = nsteps;
    a.ahat = m.ahat;
    a.chat = m.chat64;
    a.tau = m.d.tau;
    a.beta1 = m.d.beta1;
    a.beta2 = m.d.beta2;
    a.cF = m.d.c_F;
    for (size_t o = 0; o < ns; o += 65535) {
        a.s0 = o;
        active_set_kernel<<<(unsigned)std::min<size_t>(65535, ns - o), AS_NT, 0, st>>>(a);
        MFMC_LAUNCHED("active_set launch 1");
    }
    return MFMC_OK;
}

}  // namespace mfmc
