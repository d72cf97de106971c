/*
 * mfmc.h - C ABI of libmfmc: batched GPU time integration of the nonlocal,
 * non-mass-conserving Cahn-Hilliard model with obstacle potential, and the
 * multifidelity Monte Carlo (MFMC) estimator on top (arXiv 2310.10750).
 *
 * Conventions shared by every call:
 *   - Every call returns an mfmc_status.  No C++ exception crosses this boundary.
 *     On failure, mfmc_last_error() returns a message for the calling thread.
 *   - Handles (mfmc_model*, mfmc_server*) are owned by the library and released by
 *     the matching *_destroy call.  All other buffers are owned by the caller.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA device
 *     memory of the current device.  `stream` is a cudaStream_t (NULL = default
 *     stream).  Calls with device pointers are asynchronous on `stream`; calls with
 *     host output pointers return after the result has been copied back.
 *   - Fields are FP32, row-major [sample][y][x] with x fastest, n*n values each.
 *   - A device-side wait that runs out of its iteration limit, or a beta2 > 0 Newton
 *     iteration that reaches its bound, sets the model's status flag; the calls that wait
 *     for their results (mfmc_solve_batch and the mixed batch) then return
 *     MFMC_ETIMEOUT.  The context stays usable.
 */
#ifndef MFMC_H
#define MFMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MFMC_OK = 0,
    MFMC_EINVAL = 1,     /* invalid argument or descriptor                         */
    MFMC_ENOMEM = 2,     /* device or host allocation failed                       */
    MFMC_ECUDA = 3,      /* a CUDA runtime call failed                             */
    MFMC_ETIMEOUT = 4,   /* a bounded device-side wait gave up                     */
    MFMC_EBUDGET = 5,    /* the MFMC budget admits no subset (Section 4)           */
    MFMC_EBUSY = 6,      /* serving: the request is not finished yet               */
    MFMC_ENOTFOUND = 7   /* serving: unknown ticket                                */
} mfmc_status;

/* Kernel gamma of Eq. (nonl_operator).
 *   CONSTANT: gamma = 8 eps^2 / (pi delta^4) on the disc |z| <= delta, the constant
 *             whose second moment is 4 eps^2, so that L u -> -eps^2 Laplace u as
 *             delta -> 0 (the scaling Section 4 states for its kernel).
 *   GAUSSIAN: Eq. (kernel_gauss), 4 eps^2 / (pi s^4) exp(-|z|^2 / s^2), s = delta_hf/3,
 *             truncated at delta.  The printed prefactor has s^3; s^4 is the value
 *             with the same second moment and the paper's c_gamma ~ 36 eps^2/delta^2. */
typedef enum { MFMC_KERNEL_CONSTANT = 0, MFMC_KERNEL_GAUSSIAN = 1 } mfmc_kernel;

/* Boundary of the lattice Omega.  PERIODIC: the unit torus.  COLLAR: the volume-constrained
 * form of Section 2 -- the operator of Eq. (nonl_operator) integrates over Omega together
 * with the interaction collar Omega_I of width delta around it, and the collar holds the
 * fixed value bc_value (the paper leaves the collar data open; a constant is this library's
 * reading).  COLLAR runs on the TMA prefix kernels and the generic kernel (plain / direct
 * forms); the resident, row-streaming and staged-tile kernels, the mixed-fidelity call and
 * the allocation-free solve are periodic only. */
typedef enum { MFMC_BC_PERIODIC = 0, MFMC_BC_COLLAR = 1 } mfmc_boundary;

/* Initial field built on the device from a 64-bit seed (SplitMix64, one counter per
 * draw: draw i of stream k is output number k*2^32 + i + 1 of the sequence started at
 * the seed).
 *   UNIFORM:        u0 i.i.d. U[-ic_amp, ic_amp]                            (stream 1)
 *   SMOOTHED_GAUSS: ic_amp * N(0,1) noise (Box-Muller), averaged with the four
 *                   periodic neighbours, clipped to [-1, 1]                 (stream 1)
 *   NUCLEI:         Eq. (ic), four nuclei of phase -1 at (0.25,0.5), (0.75,0.5),
 *                   (0.5,0.25), (0.5,0.75) shifted by eta_i, depth mu_i; theta drawn
 *                   from U[0.9,1] x U[-0.025,0.025]^2 (stream 2) unless given; clipped.
 * Fields are built in FP64 and rounded to FP32. */
typedef enum { MFMC_IC_UNIFORM = 0, MFMC_IC_SMOOTHED_GAUSS = 1, MFMC_IC_NUCLEI = 2 } mfmc_ic;

/* Disc-sum algorithm of the step kernel. AUTO lets the autotuner pick and cache. */
typedef enum {
    MFMC_ALGO_AUTO = 0,
    MFMC_ALGO_DIRECT = 1,      /* sum over every disc point                       */
    MFMC_ALGO_PREFIX = 2,      /* in-register row prefix sums: O(R) adds per point */
    MFMC_ALGO_PREFIX_KAHAN = 3,/* prefix form with compensated accumulation       */
    MFMC_ALGO_RESIDENT = 4,    /* whole field held in shared memory for all steps */
    MFMC_ALGO_PLAIN = 5,       /* reference form: one sample per launch, direct   */
    MFMC_ALGO_PREFIX_TMA = 6,  /* prefix form, persistent CTAs, TMA double-buffered
                                  tiles of a ghost-framed field                   */
    MFMC_ALGO_ROWS = 7         /* row streaming: one CTA per SM walks its share of the
                                  batch's rows (groups of 2048/n samples) down through a ring of
                                  TMA chunks of whole rows; a warp takes a 128-column strip
                                  of one sample, a lane 4 columns with a ring of 2R+1
                                  accumulators, every staged row summed once per segment
                                  (constant kernel, R in {2,4,6,8}, n % 128 == 0)  */,
    MFMC_ALGO_FFT = 8          /* spectral form of the disc sum: cuFFT transforms (a library,
                                  loaded at run time) of each field, a product with the
                                  transform of the disc weights and the fused update; cost
                                  independent of the horizon; any kernel and radius,
                                  periodic boundary only; a comparison point for very large
                                  horizons that AUTO does not pick */,
    MFMC_ALGO_ACTIVE_SET = 9   /* the beta2 > 0 step: per step the explicit convolution (FP64;
                                  direct below 100 disc points, else spectral: by the solver's
                                  own transforms for even n <= 128 whose odd part factors into
                                  3, 5, 7 and 11, by cuFFT otherwise), then a semismooth Newton
                                  (primal-dual active-set) solve of the resolvent equation,
                                  started from the previous step's solution: FP64 fields and
                                  residual, each correction by FP32 CG preconditioned with a
                                  multigrid V-cycle; one CTA per sample; the only algorithm for
                                  beta2 > 0 (AUTO picks it), periodic only */,
    MFMC_ALGO_WEIGHTED = 10,   /* register-tiled weighted disc sum over TMA tiles: any radial
                                  kernel (the Gaussian's fastest own path), integer delta/h,
                                  either boundary; |D| FMAs per point without the prefix
                                  form's shortcut, so the constant kernel prefers PREFIX_TMA */
    MFMC_ALGO_SPECTRAL = 11    /* spectral form of the disc sum on this library's own FFT
                                  kernels: per step a column pass (FFT over y, product with the
                                  real transform of the disc weights, inverse) and a row pass
                                  (inverse row FFT, update, forward row FFT of the new rows);
                                  n = 1024 in two launches per step; n = 64 and 128 in one
                                  launch for the whole solve with the fields in shared memory
                                  (register transforms); any other even n <= 128 whose odd part
                                  is a product of 3, 5, 7 and 11 (the paper's h = 1/88) the same
                                  way with mixed-radix transforms; cost independent of the
                                  horizon; any kernel and radius, periodic boundary,
                                  beta2 = 0; AUTO considers it */
} mfmc_algo;

/* One fidelity of the model (Section 2, Section 4).  The lattice is n x n on the unit
 * torus, h = 1/n; the disc of the nodal quadrature is D = { z : |z| <= delta/h }.
 * R = floor(delta/h) must satisfy 1 <= R <= 32 and 2R + 1 <= n; n % 4 == 0 and n >= 8.
 * A non-integer delta/h (the paper's h = 1/88, delta = 0.1875 gives 16.5) is served by the
 * generic kernel only (MFMC_ALGO_PLAIN / DIRECT, which AUTO then picks).  beta2 = 0 is the
 * nonlocal Allen-Cahn limit of Eq. (nonl_CH_nm), whose step is the pointwise projection onto
 * [-1, 1] (every kernel); beta2 > 0 (the paper's 0.05) couples the step through the 5-point
 * Laplacian and is solved by MFMC_ALGO_ACTIVE_SET. */
typedef struct {
    int n;                 /* lattice points per side                              */
    double delta;          /* horizon                                              */
    mfmc_kernel kernel;
    double delta_hf;       /* Gaussian width reference (kernel GAUSSIAN only)      */
    double eps;            /* interface parameter eps (nominal)                    */
    double eps_lo, eps_hi; /* if eps_hi > eps_lo: per-sample eps ~ U[eps_lo,eps_hi]
                              drawn from stream 0 of the seed                     */
    double c_F;            /* obstacle potential constant, Eq. (potential_obstacle) */
    double beta1, beta2;   /* Eq. (nonl_CH_nm); beta1 > 0, beta2 >= 0 (beta2 > 0:
                              MFMC_ALGO_ACTIVE_SET, periodic lattice only)          */
    double tau;            /* time step                                            */
    int nsteps;            /* number of steps, T = nsteps * tau                    */
    mfmc_boundary bc;
    mfmc_ic ic;
    double ic_amp;         /* amplitude / standard deviation of the noise ICs      */
    int ic_base_n;         /* noise ICs: lattice the random field is drawn on
                              (0 = n).  A multiple b*n: u0 at a node is the mean of
                              the b x b block of base-lattice IC values, so models
                              of different n share one random input per seed.     */
    mfmc_algo algo;
    double bc_value;       /* COLLAR: the fixed value of u on the collar, in [-1, 1] */
} mfmc_model_desc;

/* Per-sample parameters (all optional).  eps <= 0 means "from the model" (the nominal
 * eps, or the per-sample draw when the model has an eps range).  has_theta = 0 draws
 * theta = (mu_i, eta_i) of Eq. (ic) from the seed.  nsteps <= 0 means the model's
 * number of steps (mfmc_solve_batch and the server honour a per-sample value). */
typedef struct {
    double eps;
    int has_theta;
    double mu[4];
    double eta[4][2];
    int nsteps;
} mfmc_sample_params;

/* Derived constants of a model (nominal eps). */
typedef struct {
    int R;                 /* delta / h                                            */
    int disc_points;       /* |D| = #{z in Z^2 : |z| <= R}                          */
    double c_gamma;        /* sum_z h^2 gamma(|z| h), the lattice c_gamma           */
    double xi;             /* c_gamma - c_F, Eq. (xi_constant)                      */
    int algo;              /* mfmc_algo the solver uses for this model             */
    size_t field_bytes;    /* n * n * 4                                             */
    int tile_variant;      /* tile shape of the TMA kernel (0..10) the solver uses */
    int band_height;       /* rows per work range of the row-streaming kernel
                              (0: the batch's rows split evenly over the warps)     */
    int columns_per_thread;/* columns per thread of the row-streaming kernel (4)   */
} mfmc_model_info;

typedef struct mfmc_model mfmc_model;
typedef struct mfmc_server mfmc_server;

/* Library version string; never NULL. */
const char *mfmc_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *mfmc_last_error(void);

/* Per-work-item trace (tracing support; the paper has no counterpart).  When on, the kernels
 * that take work items from a queue append one record per item to a ring in device memory:
 * kind 1 = an item (the whole solve of one sample, or of four on n = 64) of the resident spectral queue
 * (mfmc_solve_batch_mixed on small lattices, MFMC_ALGO_SPECTRAL outside n = 64, 128, 1024),
 * item = its ticket in the launch's queue; kind 2 = an item (one tile of one sample) of the
 * mixed-fidelity step queue, item = its ticket, step = the time step; kind 3 = one sample of
 * the beta2 > 0 solver, item = its index in the batch, step = the steps that launch ran.  t0_ns and
 * t1_ns are the GPU's global timer (ns) when the item started and ended, sm the SM that ran it. */
typedef struct {
    uint64_t t0_ns, t1_ns;
    uint32_t item, sm, kind, step;
} mfmc_trace_record;

/* Turn tracing on for the current device with a ring of `capacity` records (0 turns it off
 * and frees the ring; at most 2^28).  Replaces any earlier ring after waiting for the device.
 * Without this call, the environment variable MFMC_TRACE=<capacity> turns tracing on at the
 * first traced launch on each device.  Tracing changes no result; each record costs its kernel
 * one atomic add and one 32-byte store.  MFMC_EINVAL for a capacity above 2^28. */
mfmc_status mfmc_trace_enable(size_t capacity);

/* Wait for the current device, copy up to `max` of the records written since the last read
 * into out[] (host), oldest first, and empty the ring.  *n_out: records copied; *dropped_out:
 * records written but not copied (overwritten after the ring filled, or beyond max).  Either
 * pointer may be NULL.  MFMC_EINVAL when tracing is off on the current device. */
mfmc_status mfmc_trace_read(mfmc_trace_record *out, size_t max, size_t *n_out, uint64_t *dropped_out);

/* Validate a descriptor and create a model handle (host-side only; no device work).
 * Returns MFMC_EINVAL for: NULL pointers, n % 4 != 0 or n outside [8, 16384],
 * floor(delta/h) outside [1, 32] or a disc wider than n, tau <= 0, beta1 <= 0, beta2 < 0,
 * beta2 > 0 off the periodic lattice, eps <= 0 (without a valid eps range), c_F < 0,
 * nsteps < 0, an unknown kernel/ic/algo/bc, a collar value outside [-1, 1], a GAUSSIAN
 * kernel with delta_hf <= 0, or an algo that cannot run the model. */
mfmc_status mfmc_model_create(const mfmc_model_desc *desc, mfmc_model **out);

/* Release a model handle (NULL is ignored). */
void mfmc_model_destroy(mfmc_model *model);

/* Derived constants of a model. */
mfmc_status mfmc_model_query(const mfmc_model *model, mfmc_model_info *out);

/* Iteration totals of the model's last beta2 > 0 solve (MFMC_ALGO_ACTIVE_SET), summed over
 * its samples and steps: newton_iters = Newton residual evaluations, cg_iters = FP32 CG
 * iterations (one multigrid V-cycle each).  Reads device memory: synchronise the stream of
 * that solve first.  Zeros for a model that has run no such solve.  Either output may be
 * NULL. */
mfmc_status mfmc_model_solver_stats(const mfmc_model *model, uint64_t *newton_iters, uint64_t *cg_iters);

/* Iteration bounds of the beta2 > 0 solver (MFMC_ALGO_ACTIVE_SET; the paper states no solver for
 * its obstacle step, so the bounds are this library's): newton_max = semismooth Newton passes
 * per time step (default 60), cg_max = FP32 CG iterations per Newton correction (default 500);
 * 0 restores a default.  A step that reaches the Newton bound stops the sample's solve and sets
 * the model's status flag, so mfmc_solve_batch returns MFMC_ETIMEOUT; the device stays usable
 * and the next call starts with the flag cleared.  MFMC_EINVAL for values outside [0, 100000]. */
mfmc_status mfmc_model_set_iteration_limits(mfmc_model *model, int newton_max, int cg_max);

/* Pin the tile shape (0..10) of the TMA kernel instead of letting the autotuner choose
 * (for measurements and tests).  MFMC_EINVAL for an unknown variant. */
mfmc_status mfmc_model_set_tile_variant(mfmc_model *model, int variant);

/* Pin the work split of the row-streaming kernel: rows = rows per work range (>= 8; the
 * batch's rows, in (sample group, row) order, cut into ranges of that many rows that the CTAs
 * take in turn: CTA c owns ranges c, c + G, ...), or 0 for the rows split evenly over the
 * resident CTAs, halo rows counted (the default); columns_per_thread must be 4.  MFMC_EINVAL
 * otherwise. */
mfmc_status mfmc_model_set_band_height(mfmc_model *model, int rows, int columns_per_thread);

/* Host-side resolution of each sample's eps (model eps, eps range draw, or
 * params[i].eps), ns values into eps_out (host). params may be NULL. */
mfmc_status mfmc_sample_eps(const mfmc_model *model, const mfmc_sample_params *params,
                            const uint64_t *seeds, size_t ns, double *eps_out);

/* Build ns initial fields on the device from host seeds[ns] (and optional host
 * params[ns]) into device u0[ns][n][n].  Section 4, Eq. (ic) for NUCLEI. */
mfmc_status mfmc_init_fields(const mfmc_model *model, const mfmc_sample_params *params,
                             const uint64_t *seeds, size_t ns, float *u0, void *stream);

/* The hot path.  Advance ns fields of one model by model->nsteps steps of the scheme
 *   u^k = P_[-1,1]( (u^{k-1} + tau beta1 (gamma*u^{k-1} + c_F u^{k-1}))
 *                   / (1 + tau beta1 c_gamma) )
 * (Eq. (nonl_CH_nm) with beta2 = 0, implicit Euler with the convolution explicit as
 * Section 4 states, the convex part c_gamma u + dI implicit), and reduce the output of
 * interest f = (1 + mean u(T)) / 2 (Eq. (ooi)).  A model with beta2 > 0 takes the implicit
 * step of MFMC_ALGO_ACTIVE_SET instead (the same equation with the screened Laplacian
 * coupling, solved to max|F| <= 1e-11 per step).
 *   eps   device, ns per-sample eps values, or NULL for the nominal eps
 *   u0    device, [ns][n][n] FP32, read only
 *   uT    device, [ns][n][n] FP32 final fields, or NULL
 *   ubar  device, ns FP64 spatial means of u(T), or NULL
 *   ooi   device, ns FP64 outputs of interest, or NULL
 * Scratch (two field buffers for the streaming kernels) is owned by the library and
 * reused across calls.  ns == 0 is a no-op. */
mfmc_status mfmc_solve_fields(const mfmc_model *model, const double *eps, const float *u0,
                              size_t ns, float *uT, double *ubar, double *ooi, void *stream);

/* Same as mfmc_solve_fields with an explicit algorithm (for measurements and the
 * reference form MFMC_ALGO_PLAIN: one sample per launch, one launch per step). */
mfmc_status mfmc_solve_fields_algo(const mfmc_model *model, int algo, const double *eps,
                                   const float *u0, size_t ns, float *uT, double *ubar,
                                   double *ooi, void *stream);

/* Allocation-free variant of mfmc_solve_fields, for callers that cannot allocate device
 * memory while they solve (a framework that reserves all device memory up front through
 * its own allocator, or a latency-critical loop that must not synchronise on, or risk the
 * failure of, cudaMalloc).  The paper has no counterpart: this is a property of the
 * library, not of the method.
 * Same arguments and results as mfmc_solve_fields, computed with the register-tiled
 * prefix kernel; the scratch (two field buffers, coefficients, tile partials) is a fixed
 * 32 MiB device array inside the library that every GPU loading the library holds until
 * exit.  Limits: ns <= 4096, ns * n * n * 4 <= 16,482,304 bytes (e.g. 62 fields of
 * 256 x 256, 1006 fields of 64 x 64), ns * tiles <= 65536; larger batches return
 * MFMC_EINVAL with the limits in the message.  Constant kernel and R in
 * {1,2,3,4,5,6,8,11,12,16,22,24,32} only.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life of the process,
 * so make it before any stream capture, and do not use this call after cudaDeviceReset on
 * that device (the kept address would then be stale).  All calls share the one array and
 * it keeps the last call's contents; calls whose work overlaps on the GPU (other streams,
 * other threads) race on it. */
mfmc_status mfmc_solve_fields_noalloc(const mfmc_model *model, const double *eps, const float *u0,
                                      size_t ns, float *uT, double *ubar, double *ooi,
                                      void *stream);

/* The user-level batch call (Section 3 problem statement: OoI of model f_k at
 * parameter samples).  Sample i uses models[i], seeds[i] and params[i] (params may
 * be NULL); samples of different models run in the same call.  Host outputs:
 * ooi_out[ns] and, if not NULL, ubar_out[ns].  Synchronous. */
mfmc_status mfmc_solve_batch(mfmc_model *const *models, const mfmc_sample_params *params,
                             const uint64_t *seeds, size_t ns, double *ooi_out,
                             double *ubar_out);

/* The same batch call for a model hierarchy (Section 3: samples of f_1 ... f_K at
 * shared parameters), in one of two forms.
 *
 * Step queue: with at most 4 distinct models, each with the constant kernel and
 * R = delta/h in {2, 4, 8, 16}, the samples of every model that streams through HBM are
 * advanced by ONE kernel launch per time step: the (model, sample, tile) items of those models
 * form one work queue, fine model first, that persistent CTAs drain through an atomic ticket
 * counter.  Models whose whole field fits in shared memory (the resident kernel, n <= 128)
 * instead run all their steps in one resident launch each, on a second stream concurrent with
 * the step launches.  The fields of the queued models are bit-identical to those of the TMA
 * prefix kernel with 4 columns per thread, their OoI differs from that solve's only by the
 * FP64 summation order of the tile partials, and resident models give the resident kernel's
 * results.  The step loop is captured in a CUDA graph on the first call of a shape and
 * replayed by later calls of the same shape.
 *
 * Resident spectral queue: otherwise, when every model (at most 16) has the periodic lattice,
 * beta2 = 0, an even n <= 128 whose odd part is a product of 3, 5, 7 and 11, and any kernel and
 * horizon (the paper's nine models of Section 4 / Table 1, delta/h = 16.5 included), ONE
 * launch runs every sample's whole solve: persistent CTAs take (model, sample group) items,
 * heaviest model first, through an atomic ticket counter, and keep the fields in shared memory
 * for all steps, each item on the form MFMC_ALGO_SPECTRAL uses for its lattice (register
 * transforms on n = 64, four samples an item, and n = 128; mixed-radix transforms otherwise).
 * Results equal those of MFMC_ALGO_SPECTRAL's solves of the same samples.
 *
 * Same arguments and results as mfmc_solve_batch; every sample runs >= 1 step.  Other inputs
 * return MFMC_EINVAL.  Calls are serialised by a lock; the library keeps the batch buffers
 * until exit.  Synchronous. */
mfmc_status mfmc_solve_batch_mixed(mfmc_model *const *models, const mfmc_sample_params *params,
                                   const uint64_t *seeds, size_t ns, double *ooi_out,
                                   double *ubar_out);

/* ---------------------------------------------------------------- MFMC (Section 3) */

#define MFMC_MAX_MODELS 16

/* A model selection and sample allocation.  Indices are 0-based model numbers;
 * idx[0] == 0 is the high-fidelity model f_1.  Arrays are indexed by the position j
 * in the selected subset (0-based).  alpha[0] = 1. */
typedef struct {
    int K_sel;                        /* |S|                                     */
    int idx[MFMC_MAX_MODELS];         /* i_j                                     */
    double rho[MFMC_MAX_MODELS];      /* rho_{1,i_j}                             */
    double sigma[MFMC_MAX_MODELS];    /* sigma_{i_j}                             */
    double cost[MFMC_MAX_MODELS];     /* C_{i_j}                                 */
    double alpha[MFMC_MAX_MODELS];    /* Eq. (alpha)                             */
    double r[MFMC_MAX_MODELS];        /* Eq. (rk)                                */
    double m_real[MFMC_MAX_MODELS];   /* Eq. (samples) or the below-B_min branch  */
    int64_t m[MFMC_MAX_MODELS];       /* floor(m_real)                           */
    double V;                         /* Eq. (variance_reduction_ratio)          */
    double Bmin;                      /* Eq. (bmin)                              */
    double mse_theory;                /* Eq. (error_theory)                      */
    double budget;
    int below_min_budget;             /* 1 if the Section 4 branch was used      */
    int n_feasible;                   /* feasible subsets, Eqs. (conditiona/b)   */
    int n_models;                     /* K                                       */
    double rho_all[MFMC_MAX_MODELS];  /* rho_{1,k} of every model                */
    double sigma_all[MFMC_MAX_MODELS];/* sigma_k of every model                  */
    double mean_all[MFMC_MAX_MODELS]; /* pilot mean of every model               */
} mfmc_plan_t;

/* Pilot statistics in FP64 on the GPU (Section 3.1): for K models on the same n
 * pilot samples, device ooi[K][n] -> host mean[K], sigma[K] (n-1 convention) and
 * rho[K] = Cov(f_1, f_k) / (sigma_1 sigma_k).  Deterministic reduction order. */
mfmc_status mfmc_pilot_stats(int K, int n, const double *ooi_dev, double *mean,
                             double *sigma, double *rho, void *stream);

/* Model selection and allocation (Section 3): pilot OoIs (host [K][n_pilot], model 0
 * is f_1), costs (host [K], any unit consistent with budget), budget B.
 * Policies: 0 smallest V with B >= B_min, else the smallest-V subset that admits the
 * below-minimum-budget branch of Section 4; 1 smallest V regardless of B_min (Case 1);
 * 2 smallest B_min (Case 3); 3 the explicit subset (explicit_idx[0..explicit_len-1],
 * starting with 0).  Returns MFMC_EBUDGET when no subset fits B (the Section 4
 * requirement B >= sum_l l C_{i_l}), and when no subset with a surrogate meets
 * Eq. (conditionb) (policies 0-2: nothing to select).  With K = 1 the plan is plain Monte
 * Carlo. */
mfmc_status mfmc_plan(int K, int n_pilot, const double *pilot_ooi, const double *costs,
                      double budget, int policy, const int *explicit_idx, int explicit_len,
                      mfmc_plan_t *out);

/* mfmc_plan from statistics that are already known (a previous study's table, such as
 * the paper's Table 1), host only, no device work: rho[K] = rho_{1,k} (rho[0] is f_1's
 * own, 1), sigma[K] > 0, costs[K] > 0 (host), budget, policy and explicit subset as for
 * mfmc_plan; the plan's mean_all is zero.  MFMC_EINVAL for a NULL pointer, K outside
 * [1, 16], |rho| > 1 or a non-finite value; MFMC_EBUDGET as for mfmc_plan. */
mfmc_status mfmc_plan_from_stats(int K, const double *rho, const double *sigma, const double *costs,
                                 double budget, int policy, const int *explicit_idx, int explicit_len,
                                 mfmc_plan_t *out);

/* Eq. (MFMC_estimator) in FP64 on the GPU: ooi[j] (host) holds model i_j on the
 * shared sample sequence, at least m_j values; Q^{(i_j)}_m is the mean of the first m.
 * Writes the estimate to *estimate (host). */
mfmc_status mfmc_estimate(const mfmc_plan_t *plan, const double *const *ooi,
                          double *estimate);

/* Device variant: ooi_dev[j] device pointers, estimate_dev a device double. */
mfmc_status mfmc_estimate_device(const mfmc_plan_t *plan, const double *const *ooi_dev,
                                 double *estimate_dev, void *stream);

/* Pilot -> plan -> allocated solves -> estimate, all samples on the GPU.
 * models[K] (models[0] = f_1); pilot seeds are seed_base + 0..n_pilot-1 and the
 * estimation seeds are seed_base + n_pilot + 0..m_j-1 (nested, disjoint from the
 * pilot).  costs (host [K]) may be NULL: then each model's cost is measured as GPU
 * seconds per sample from the pilot solve.  Outputs plan_out and *estimate (host). */
mfmc_status mfmc_run(mfmc_model *const *models, int K, int n_pilot, double budget,
                     int policy, uint64_t seed_base, const double *costs,
                     mfmc_plan_t *plan_out, double *estimate);

/* ---------------------------------------------------------------- serving */

/* Serving statistics.  Latencies are submit-to-completion wall seconds. */
typedef struct {
    uint64_t submitted, completed, rejected;
    double p50_latency_s, p99_latency_s, mean_latency_s;
    double samples_per_s;          /* completed / (last completion - first submit) */
    size_t peak_bytes;             /* peak device bytes held by admitted requests  */
    int peak_inflight;
} mfmc_server_stats;

/* Continuous-batching request loop on one GPU: a host thread admits submitted solve
 * requests while their fields fit in hbm_budget_bytes and fewer than max_slots are in
 * flight, keeps their fields resident on the device, and advances all admitted
 * requests together between admissions, so requests that arrive while others run join
 * the work already on the GPU. */
mfmc_status mfmc_server_create(size_t hbm_budget_bytes, int max_slots, mfmc_server **out);

/* Queue one solve (model, optional params, seed); returns a ticket.  The model must
 * outlive the request.  Thread-safe. */
mfmc_status mfmc_submit(mfmc_server *srv, const mfmc_model *model,
                        const mfmc_sample_params *params, uint64_t seed, uint64_t *ticket);

/* MFMC_OK with the result once done (the ticket is then released), MFMC_EBUSY while
 * queued or running, MFMC_ENOTFOUND for an unknown ticket. */
mfmc_status mfmc_poll(mfmc_server *srv, uint64_t ticket, double *ooi, double *latency_s);

/* When a finished request was submitted, admitted (its cohort queued on the GPU) and found
 * complete, in seconds since the server was created (host outputs, each may be NULL).  Kept
 * after mfmc_poll, until mfmc_server_destroy.  MFMC_EBUSY while the request runs,
 * MFMC_ENOTFOUND for a ticket the server never issued.  Serving is not in the paper: this
 * shows which requests ran on the device at the same time. */
mfmc_status mfmc_request_times(mfmc_server *srv, uint64_t ticket, double *submit_s, double *admit_s,
                               double *done_s);

/* Block until every submitted request has completed. */
mfmc_status mfmc_server_drain(mfmc_server *srv);

mfmc_status mfmc_server_get_stats(mfmc_server *srv, mfmc_server_stats *out);

/* Stop the loop thread and release device memory (NULL is ignored). */
void mfmc_server_destroy(mfmc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* MFMC_H */
