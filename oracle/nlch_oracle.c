/*
 * Oracle (test infrastructure only): a plain, slow FP64 CPU implementation of the
 * discretised nonlocal Cahn-Hilliard model with obstacle potential (Section 2,
 * Eq. (nonl_CH_nm) with beta2 = 0, Eq. (nonl_operator), Eq. (potential_obstacle))
 * and of the output of interest (Section 4, Eq. (ooi)).
 *
 * Only tests, the package smoke check and the CPU-baseline leg of the benchmark may
 * load this code.  It shares nothing with the CUDA library: its random-number
 * generator, initial conditions, kernel weights, time step and reductions are
 * written out here on their own from the paper and from the published SplitMix64
 * definition.
 *
 * Discretisation (Section 4 names P1 finite elements with mass lumping, implicit
 * Euler in time and an explicit convolution; the FE assembly itself is in papers the
 * text only cites).  The reading used here: a periodic n x n lattice with h = 1/n,
 * nodal quadrature of the convolution,
 *     (gamma * u)_i = sum_{z in D} h^2 gamma(|z| h) u_{i+z},
 *     D = { z in Z^2 : |z|^2 <= (delta/h)^2 },
 *     c_gamma = sum_{z in D} h^2 gamma(|z| h),
 * and per step the convex part c_gamma u + dI(u) taken implicitly while the
 * convolution and the concave part -c_F u are explicit:
 *     (u^k - u^{k-1})/tau + beta1 w^k = 0,
 *     w^k in c_gamma u^k - (gamma * u^{k-1} + c_F u^{k-1}) + dI(u^k).
 * With beta2 = 0 this inclusion is pointwise and its unique solution is
 *     u^k = P_[-1,1]( (u^{k-1} + tau beta1 (gamma*u^{k-1} + c_F u^{k-1}))
 *                     / (1 + tau beta1 c_gamma) ).
 *
 * Every routine is written for clarity: direct loops, modular indexing, FP64
 * throughout, sequential sums in index order.  OpenMP (when compiled in) only splits
 * independent output rows; each output is computed by one thread in a fixed order,
 * so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by the     */
/* golden-ratio increment and each output is the state passed through a        */
/* fixed 64-bit finaliser.  Output number pos (pos >= 1) of the sequence that  */
/* starts from state `seed` is mix(seed + pos * increment).                    */
/* ------------------------------------------------------------------------- */
static const uint64_t ORC_SM64_INC = 0x9E3779B97F4A7C15ULL;

static uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t pos) {
    return orc_mix64(seed + pos * ORC_SM64_INC);
}

/* Draw `idx` of stream `stream` for `seed`: output number stream*2^32 + idx + 1. */
uint64_t orc_draw(uint64_t seed, uint32_t stream, uint32_t idx) {
    return orc_splitmix64(seed, ((uint64_t)stream << 32) + (uint64_t)idx + 1ULL);
}

/* Uniform double in [0, 1): the top 53 bits of the draw times 2^-53. */
double orc_uniform(uint64_t seed, uint32_t stream, uint32_t idx) {
    return (double)(orc_draw(seed, stream, idx) >> 11) * 0x1p-53;
}

/* Standard normal from two uniforms by the Box-Muller transform (Box & Muller 1958). */
double orc_normal(uint64_t seed, uint32_t stream, uint32_t idx) {
    double u1 = 1.0 - orc_uniform(seed, stream, 2u * idx);      /* in (0, 1] */
    double u2 = orc_uniform(seed, stream, 2u * idx + 1u);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------- */
/* The horizon disc and the kernel weights                                    */
/* ------------------------------------------------------------------------- */

/* Lattice offsets inside the disc |z| <= rad (rad = delta/h), in row-major order of
 * (dy, dx).  Returns the count; writes at most `cap` entries. */
int orc_disc(double rad, int *dx, int *dy, int cap) {
    int Rc = (int)floor(rad + 1e-9);
    double r2 = rad * rad * (1.0 + 1e-12);
    int count = 0;
    for (int j = -Rc; j <= Rc; ++j)
        for (int i = -Rc; i <= Rc; ++i)
            if ((double)(i * i + j * j) <= r2) {
                if (count < cap) { dx[count] = i; dy[count] = j; }
                ++count;
            }
    return count;
}

/* Kernel value gamma(r) for the two kernels of the model.
 * kind 0, constant on the disc, scaled so that L u -> -eps^2 Laplace u as delta -> 0
 *   (the scaling stated in Section 4 for Eq. (kernel_gauss)): the second moment
 *   int |z|^2 gamma dz equals 4 eps^2, which for a constant A on B_delta gives
 *   A = 8 eps^2 / (pi delta^4).
 * kind 1, the truncated Gaussian of Eq. (kernel_gauss) with s = delta_hf/3.  The
 *   printed prefactor has s^3; s^4 is the value that gives the same second moment
 *   and reproduces the paper's own c_gamma ~ 36 eps^2/delta^2 and xi ~ 0.0253. */
double orc_gamma(int kind, double r, double eps, double delta, double delta_hf) {
    if (r > delta * (1.0 + 1e-12)) return 0.0;
    if (kind == 0) return 8.0 * eps * eps / (M_PI * pow(delta, 4));
    double s = delta_hf / 3.0;
    return 4.0 * eps * eps / (M_PI * pow(s, 4)) * exp(-(r * r) / (s * s));
}

/* Quadrature weights w_z = h^2 gamma(|z| h) for the disc offsets; returns c_gamma. */
double orc_weights(int kind, int n, double delta, double eps, double delta_hf,
                   const int *dx, const int *dy, int count, double *w) {
    double h = 1.0 / n, cg = 0.0;
    for (int k = 0; k < count; ++k) {
        double r = h * sqrt((double)(dx[k] * dx[k] + dy[k] * dy[k]));
        w[k] = h * h * orc_gamma(kind, r, eps, delta, delta_hf);
        cg += w[k];
    }
    return cg;
}

static inline int orc_wrap(int a, int n) { int m = a % n; return m < 0 ? m + n : m; }

/* (gamma * u)_i on the periodic lattice, direct sum over the disc. */
void orc_convolve(int n, const double *u, const int *dx, const int *dy, const double *w,
                  int count, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double s = 0.0;
            for (int k = 0; k < count; ++k)
                s += w[k] * u[orc_wrap(y + dy[k], n) * n + orc_wrap(x + dx[k], n)];
            out[y * n + x] = s;
        }
}

/* Nonlocal operator of Eq. (nonl_operator) in its difference form,
 * (L u)_i = sum_z w_z (u_i - u_{i+z}); it vanishes exactly on constant fields. */
void orc_apply_L(int n, const double *u, const int *dx, const int *dy, const double *w,
                 int count, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double ui = u[y * n + x], s = 0.0;
            for (int k = 0; k < count; ++k)
                s += w[k] * (ui - u[orc_wrap(y + dy[k], n) * n + orc_wrap(x + dx[k], n)]);
            out[y * n + x] = s;
        }
}

/* Same operator without wrap-around, evaluated only at interior points whose disc
 * stays inside the array (entries closer than Rc to an edge are set to NAN).  Used
 * to check the closed form on non-periodic fields such as x^2. */
void orc_apply_L_open(int n, const double *u, const int *dx, const int *dy, const double *w,
                      int count, int Rc, double *out) {
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            if (y < Rc || y >= n - Rc || x < Rc || x >= n - Rc) { out[y * n + x] = NAN; continue; }
            double ui = u[y * n + x], s = 0.0;
            for (int k = 0; k < count; ++k) s += w[k] * (ui - u[(y + dy[k]) * n + x + dx[k]]);
            out[y * n + x] = s;
        }
}

/* One time step (beta2 = 0): explicit convolution, implicit convex part, and the
 * resolvent of the indicator (the projection onto [-1, 1]). */
void orc_step(int n, const double *u, double *unew, const int *dx, const int *dy,
              const double *w, int count, double cgam, double cF, double tau, double beta1) {
    double denom = 1.0 + tau * beta1 * cgam;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double conv = 0.0;
            for (int k = 0; k < count; ++k)
                conv += w[k] * u[orc_wrap(y + dy[k], n) * n + orc_wrap(x + dx[k], n)];
            double ui = u[y * n + x];
            double v = (ui + tau * beta1 * (conv + cF * ui)) / denom;
            unew[y * n + x] = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
        }
}

/* ------------------------------------------------------------------------- */
/* Volume-constrained boundary (Section 2: the operator integrates over        */
/* Omega together with the interaction collar Omega_I of width delta around it; */
/* the paper leaves the data on Omega_I open).  Reading: Omega is the n x n     */
/* lattice without wrap-around, every lattice point outside it within the      */
/* horizon belongs to the collar and holds the fixed value uI, and the scheme  */
/* is unchanged otherwise.  c_gamma stays the full-disc sum, so L vanishes on  */
/* u = uI everywhere.  The collar value of a point is read by orc_collar_at.   */
/* ------------------------------------------------------------------------- */
static inline double orc_collar_at(int n, const double *u, int y, int x, double uI) {
    if (y < 0 || y >= n || x < 0 || x >= n) return uI;
    return u[y * n + x];
}

/* (gamma * u)_i with the collar: direct sum over the disc. */
void orc_convolve_collar(int n, const double *u, const int *dx, const int *dy, const double *w,
                         int count, double uI, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double s = 0.0;
            for (int k = 0; k < count; ++k) s += w[k] * orc_collar_at(n, u, y + dy[k], x + dx[k], uI);
            out[y * n + x] = s;
        }
}

/* (L u)_i = sum_z w_z (u_i - u_{i+z}) with the collar. */
void orc_apply_L_collar(int n, const double *u, const int *dx, const int *dy, const double *w,
                        int count, double uI, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double ui = u[y * n + x], s = 0.0;
            for (int k = 0; k < count; ++k) s += w[k] * (ui - orc_collar_at(n, u, y + dy[k], x + dx[k], uI));
            out[y * n + x] = s;
        }
}

/* One time step (beta2 = 0) with the collar: as orc_step, the convolution reads uI
 * outside Omega. */
void orc_step_collar(int n, const double *u, double *unew, const int *dx, const int *dy,
                     const double *w, int count, double cgam, double cF, double tau, double beta1,
                     double uI) {
    double denom = 1.0 + tau * beta1 * cgam;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double conv = 0.0;
            for (int k = 0; k < count; ++k) conv += w[k] * orc_collar_at(n, u, y + dy[k], x + dx[k], uI);
            double ui = u[y * n + x];
            double v = (ui + tau * beta1 * (conv + cF * ui)) / denom;
            unew[y * n + x] = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
        }
}

/* Spatial mean of u: the lumped-mass integral (h^2 sum_i u_i) divided by |Omega| = 1. */
double orc_mean(int n, const double *u) {
    double s = 0.0;
    for (long i = 0; i < (long)n * n; ++i) s += u[i];
    return s / ((double)n * (double)n);
}

/* Eq. (ooi): f = (1 + mean(u)) / 2. */
double orc_ooi(int n, const double *u) { return 0.5 * (1.0 + orc_mean(n, u)); }

/* Discrete energy E_h(u) = h^2 [ 1/4 sum_i sum_z w_z (u_i - u_{i+z})^2
 *                              + sum_i (c_F/2)(1 - u_i^2) ]  for |u_i| <= 1
 * (the nonlocal free energy whose gradient is L_h u + dF_obs(u)). */
double orc_energy(int n, const double *u, const int *dx, const int *dy, const double *w,
                  int count, double cF) {
    double h2 = 1.0 / ((double)n * n), e_int = 0.0, e_pot = 0.0;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double ui = u[y * n + x];
            for (int k = 0; k < count; ++k) {
                double d = ui - u[orc_wrap(y + dy[k], n) * n + orc_wrap(x + dx[k], n)];
                e_int += w[k] * d * d;
            }
            e_pot += 0.5 * cF * (1.0 - ui * ui);
        }
    return h2 * (0.25 * e_int + e_pot);
}

/* Symbol of L_h on the Fourier mode exp(i 2 pi (p x + q y)):
 *   c_gamma - sum_z w_z cos(2 pi (p dx + q dy) / n). */
double orc_symbol(int n, int p, int q, const int *dx, const int *dy, const double *w, int count) {
    double s = 0.0, cg = 0.0;
    for (int k = 0; k < count; ++k) {
        cg += w[k];
        s += w[k] * cos(2.0 * M_PI * (double)(p * dx[k] + q * dy[k]) / (double)n);
    }
    return cg - s;
}

/* ------------------------------------------------------------------------- */
/* Initial conditions (all built in FP64 and then rounded to FP32 values)       */
/* ------------------------------------------------------------------------- */

static double orc_clip1(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

/* ic 0: i.i.d. uniform on [-amp, amp] (stream 1, one draw per node). */
/* ic 1: Gaussian noise amp * N(0,1) (stream 1, two draws per node), averaged with its
 *       four periodic lattice neighbours, (c + left + right + down + up)/5 in that order,
 *       then clipped to [-1, 1]. */
/* For ic 0 and 1 the random field is drawn on a base lattice of base_n = b*n points per
 * side (b >= 1); the node (y, x) of the n-lattice takes the mean of the b x b base
 * nodes (b y + a, b x + c), a, c in [-(b/2), b - b/2), summed a-major in FP64.  With
 * b = 1 this is the field itself.  Models of different n then share one random input. */
/* ic 2: Eq. (ic), four nuclei: u0 = 1 - 2 sum_i mu_i exp(-36 |x - xbar_i - eta_i|^2),
 *       with the minimum-image distance on the unit torus, nodes at (j h, i h), and
 *       the result clipped to [-1, 1].  theta = (mu_i, eta_i) is passed in. */
static void orc_noise_field(int N, int ic, double amp, uint64_t seed, double *f) {
    long NN = (long)N * N;
    if (ic == 0) {
        for (long i = 0; i < NN; ++i) f[i] = amp * (2.0 * orc_uniform(seed, 1, (uint32_t)i) - 1.0);
        return;
    }
    double *z = (double *)malloc(sizeof(double) * NN);
    for (long i = 0; i < NN; ++i) z[i] = amp * orc_normal(seed, 1, (uint32_t)i);
    for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
            double s = z[y * N + x];
            s += z[y * N + orc_wrap(x - 1, N)];
            s += z[y * N + orc_wrap(x + 1, N)];
            s += z[orc_wrap(y - 1, N) * N + x];
            s += z[orc_wrap(y + 1, N) * N + x];
            f[y * N + x] = orc_clip1(s / 5.0);
        }
    free(z);
}

/* Block mean of a base-lattice field f (B x B, B = b n) onto the n-lattice: node (y, x)
 * takes the mean of the b x b base nodes (b y + a, b x + c), a, c in [-(b/2), b - b/2)
 * (periodic), summed a-major in FP64. */
void orc_block_mean(int n, int B, const double *f, double *u) {
    int b = B / n;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double s = 0.0;
            for (int a = -(b / 2); a < b - b / 2; ++a)
                for (int c = -(b / 2); c < b - b / 2; ++c)
                    s += f[orc_wrap(b * y + a, B) * B + orc_wrap(b * x + c, B)];
            u[y * n + x] = s / ((double)b * (double)b);
        }
}

void orc_initial_field(int n, int ic, double amp, uint64_t seed, const double *mu,
                       const double *eta, int base_n, double *u0) {
    long N = (long)n * n;
    if (ic == 0 || ic == 1) {
        int B = base_n > 0 ? base_n : n;
        double *f = (double *)malloc(sizeof(double) * (size_t)B * B);
        orc_noise_field(B, ic, amp, seed, f);
        orc_block_mean(n, B, f, u0);
        free(f);
    } else {
        static const double cx[4] = {0.25, 0.75, 0.5, 0.5};
        static const double cy[4] = {0.5, 0.5, 0.25, 0.75};
        double h = 1.0 / n;
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double s = 0.0;
                for (int k = 0; k < 4; ++k) {
                    double ddx = x * h - (cx[k] + eta[2 * k]);
                    double ddy = y * h - (cy[k] + eta[2 * k + 1]);
                    ddx -= floor(ddx + 0.5);
                    ddy -= floor(ddy + 0.5);
                    s += mu[k] * exp(-36.0 * (ddx * ddx + ddy * ddy));
                }
                u0[y * n + x] = orc_clip1(1.0 - 2.0 * s);
            }
    }
    for (long i = 0; i < N; ++i) u0[i] = (double)(float)u0[i];
}

/* theta for the nuclei IC drawn from the seed (stream 2): mu_i ~ U[0.9, 1],
 * eta_i ~ U[-0.025, 0.025]^2, the parameter domain of Eq. (ic). */
void orc_draw_theta(uint64_t seed, double *mu, double *eta) {
    for (int k = 0; k < 4; ++k) {
        mu[k] = 0.9 + 0.1 * orc_uniform(seed, 2, 3u * k);
        eta[2 * k] = -0.025 + 0.05 * orc_uniform(seed, 2, 3u * k + 1u);
        eta[2 * k + 1] = -0.025 + 0.05 * orc_uniform(seed, 2, 3u * k + 2u);
    }
}

/* Per-sample interface parameter: eps itself when eps_hi <= eps_lo, else a uniform
 * draw on [eps_lo, eps_hi] from stream 0 of the seed. */
double orc_sample_eps(uint64_t seed, double eps, double eps_lo, double eps_hi) {
    if (!(eps_hi > eps_lo)) return eps;
    return eps_lo + (eps_hi - eps_lo) * orc_uniform(seed, 0, 0);
}

/* Full solve of one sample: nsteps steps from u (overwritten with u(T)).  Returns
 * the spatial mean of u(T); the output of interest is (1 + mean)/2. */
double orc_solve(int n, double *u, int nsteps, const int *dx, const int *dy, const double *w,
                 int count, double cgam, double cF, double tau, double beta1) {
    long N = (long)n * n;
    double *a = u, *b = (double *)malloc(sizeof(double) * N);
    for (int k = 0; k < nsteps; ++k) {
        orc_step(n, a, b, dx, dy, w, count, cgam, cF, tau, beta1);
        double *t = a; a = b; b = t;
    }
    if (a != u) { memcpy(u, a, sizeof(double) * N); b = a; }
    free(b);
    return orc_mean(n, u);
}

/* Full solve of one sample with the collar (see orc_step_collar). */
double orc_solve_collar(int n, double *u, int nsteps, const int *dx, const int *dy, const double *w,
                        int count, double cgam, double cF, double tau, double beta1, double uI) {
    long N = (long)n * n;
    double *a = u, *b = (double *)malloc(sizeof(double) * N);
    for (int k = 0; k < nsteps; ++k) {
        orc_step_collar(n, a, b, dx, dy, w, count, cgam, cF, tau, beta1, uI);
        double *t = a; a = b; b = t;
    }
    if (a != u) { memcpy(u, a, sizeof(double) * N); b = a; }
    free(b);
    return orc_mean(n, u);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
