// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "mfmc.h"

namespace mfmc {

constexpr int kMaxR = 32;
constexpr int kMaxNs = 1 << 24;
// default iteration bounds of the beta2 > 0 solver: Newton passes per step, FP32 CG iterations
// per Newton correction (mfmc_model_set_iteration_limits changes them per model)
constexpr int kAsNewtonMax = 60;
constexpr int kAsCgMax = 500;

// Step coefficients of one sample.  With S = sum_z what_z u_{i+z} (what_z = 1 for the
// constant kernel, the Gaussian weight / eps^2 otherwise) the update is
//   v = u + c1 * (S - c0 * u) + c2 * u,   u_new = min(1, max(-1, v)),
// where c0 = sum_z what_z, c1 = tau beta1 eps^2 ahat / (1 + tau beta1 c_gamma),
// c2 = tau beta1 c_F / (1 + tau beta1 c_gamma) and c_gamma = eps^2 ahat c0.
// This is the scheme (u + tau beta1 (gamma*u + c_F u)) / (1 + tau beta1 c_gamma)
// rearranged so that the increment is formed from small terms.
struct StepCoef {
    float c0, c1, c2, pad;
};

struct FftState;  // spectral-convolution state of the FFT path (fft_solver.cu)
void fft_release(FftState *f);
bool fft_available();
struct SpectralState;  // the own-FFT spectral path (spectral.cu)
void spectral_release(SpectralState *s);
struct Fft64State;  // FP64 spectral disc sums of the beta2 > 0 solver (fft_solver.cu)
void fft64_release(Fft64State *f);
bool fft64_available();

// A validated model: descriptor plus derived constants.
struct Model {
    mfmc_model_desc d;
    int R;                    // floor(delta / h): the disc's extent in lattice points
    int r2max;                // floor((delta / h)^2): the disc is { z : |z|^2 <= r2max }
    int integer_R;            // 1 when delta / h is an integer (every kernel); 0: generic kernel only
    int disc;                 // |D_R|
    int widths[kMaxR + 1];    // w(|dy|) = floor(sqrt(R^2 - dy^2))
    double ahat;              // gamma h^2 / eps^2 at r = 0 for the constant kernel, 1 for Gaussian
    std::vector<float> wtab;  // Gaussian: weight / eps^2 per r2 = dx^2 + dy^2 (0..R^2)
    double chat;              // sum_z what_z (FP64)
    std::vector<double> wtab64; // Gaussian: FP64 weight / eps^2 per r2 (the beta2 > 0 solver)
    double chat64 = 0.0;      // sum_z what_z of the FP64 weights
    // scratch of the beta2 > 0 solver (active_set.cu)
    double *d_wtab64 = nullptr;
    std::vector<float> wsq;   // weighted TMA form: weights by (|dy|, |dx|), zero outside the disc
    float *d_wsq = nullptr;
    double *as_buf = nullptr;
    size_t as_cap = 0;        // doubles
    int algo;                 // resolved algorithm (never AUTO after the autotuner ran)
    int tuned;                // 1 once AUTO was resolved
    // library-owned scratch, reused across calls on this model
    std::mutex mu;
    float *bufA = nullptr, *bufB = nullptr;
    size_t buf_cap = 0;       // samples
    double *partials = nullptr;
    size_t partials_cap = 0;  // doubles
    StepCoef *coef = nullptr;
    size_t coef_cap = 0;
    float *d_wtab = nullptr;
    double *eps_tmp = nullptr;
    size_t eps_cap = 0;
    uint64_t *seeds_tmp = nullptr;
    double *theta_tmp = nullptr;
    size_t seeds_cap = 0;
    // buffers of the batch call (initial fields and results), and its stream
    float *u0buf = nullptr;
    size_t u0_cap = 0;
    double *resbuf = nullptr;
    size_t res_cap = 0;
    cudaStream_t stream = nullptr;
    // ghost-framed scratch of the TMA path: [cap][P][P], P = n + 2 G, and its tensor maps
    float *padA = nullptr, *padB = nullptr;
    size_t pad_cap = 0;
    CUtensorMap mapA, mapB;
    int maps_valid = 0;
    int map_sw = 0, map_sh = 0, map_sd = 1, map_l2 = 256;  // box and L2 promotion of the tensor maps
    int tma_variant = 4;         // tile shape of the TMA kernel (autotuned; 4 is the default)
    int rows_bh = 0;             // rows per work range of the row-streaming kernel (0: even split)
    int rows_rx = 4;             // columns per thread of the row-streaming kernel
    int *d_status = nullptr;  // set by a device wait that gave up
    // CUDA graph of the last solve's launch sequence (replayed while its key matches)
    cudaGraphExec_t gexec = nullptr;
    std::vector<uintptr_t> gkey;
    int graphs_off = 0;
    FftState *fft = nullptr;  // created by the first FFT-path solve
    Fft64State *fft64 = nullptr;  // created by the first spectral beta2 > 0 solve
    SpectralState *spectral = nullptr;  // created by the first own-FFT spectral solve
    float *d_khat32 = nullptr;    // resident spectral form: K^ / n^2 at [ky][n/2 + 1] (FP32)
    float2 *d_tw32 = nullptr;     // and W_n^j, j < n
    int sr_dev = -1;              // device of those tables
    int *sr_counter = nullptr;    // its ticket counter
    double *d_khat64 = nullptr;   // beta2 > 0, own FFT: K^ / n^2 at [ky][n/2 + 1] (FP64)
    double2 *d_tw64 = nullptr;    // and W_n^j, j < n
    unsigned long long *d_as_iters = nullptr;  // Newton and CG iterations of the last beta2 > 0 solve
    int as_newton_max = kAsNewtonMax;           // iteration bounds of the beta2 > 0 solver
    int as_cg_max = kAsCgMax;
    ~Model();
};

// error helpers (thread-local message)
void set_error(const char *fmt, ...);
mfmc_status fail(mfmc_status s, const char *fmt, ...);
mfmc_status cuda_fail(cudaError_t e, const char *what);

#define MFMC_LAUNCHED(what)                                               \
    do {                                                                  \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return ::mfmc::cuda_fail(e_, what);        \
    } while (0)

#define MFMC_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::mfmc::cuda_fail(e_, #call);       \
    } while (0)

// SplitMix64, library side (Steele, Lea & Flood 2014): draw i of stream k of a seed is
// output number k * 2^32 + i + 1 of the sequence whose state starts at the seed.
__host__ __device__ inline uint64_t sm64_finalize(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t sm64_draw(uint64_t seed, uint32_t stream, uint32_t i) {
    const uint64_t pos = ((uint64_t)stream << 32) + (uint64_t)i + 1ULL;
    return sm64_finalize(seed + pos * 0x9E3779B97F4A7C15ULL);
}
__host__ __device__ inline double sm64_unit(uint64_t seed, uint32_t stream, uint32_t i) {
    return (double)(sm64_draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

// Per-sample eps on the host: params, else the model's range draw, else nominal.
double resolve_eps(const Model &m, const mfmc_sample_params *p, uint64_t seed);
// Per-sample theta (mu[4], eta[8]) on the host: params or a draw from stream 2.
void resolve_theta(const mfmc_sample_params *p, uint64_t seed, double theta[12]);

template <typename T>
mfmc_status grow_buffer(T **p, size_t *cap, size_t want) {
    if (*cap >= want && *p) return MFMC_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (want == 0) return MFMC_OK;
    cudaError_t e = cudaMalloc((void **)p, want * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc (scratch)");
    }
    *cap = want;
    return MFMC_OK;
}

// Grow the model's scratch to hold ns samples (fields + partials + coefficients).
mfmc_status ensure_scratch(Model &m, size_t ns, size_t partials_per_sample);

// kernels (launch helpers), all asynchronous on `st`
mfmc_status launch_init_fields(const Model &m, const uint64_t *seeds_dev,
                               const double *theta_dev, size_t ns, float *u0, cudaStream_t st);
mfmc_status launch_coefficients(const Model &m, const double *eps_dev, size_t ns,
                                StepCoef *coef, cudaStream_t st);
// Full solve with an explicit algorithm; scratch from the model.
mfmc_status run_solve(Model &m, int algo, const StepCoef *coef, const float *u0, size_t ns,
                      int nsteps, float *uT, double *ubar, double *ooi, cudaStream_t st);
// Buffers of one run of the TMA pipeline (model scratch, or a serving cohort's own).
struct TmaBuffers {
    float *padA = nullptr, *padB = nullptr;
    CUtensorMap mapA, mapB;
    CUtensorMap mapA1, mapB1;  // the row-streaming kernel's one-row boxes
    size_t cap = 0;
    double *partials = nullptr;
    int *status = nullptr;
};
// Tensor map of padded fields [cap][P][P] FP32 with a box of sw x sh x sd (x, y, sample) and
// L2 promotion of l2promo bytes (256, 128 or 0).
mfmc_status encode_map(CUtensorMap *map, float *base, int P, size_t cap, int sw, int sh, int sd = 1,
                       int l2promo = 256);
int tma_tiles(const Model &m, int variant, int *tiles_x);
// stream-ordered allocation on alloc_st (cudaMallocAsync) and release (cudaFreeAsync)
mfmc_status tma_alloc_buffers(const Model &m, int variant, size_t ns, TmaBuffers *b, cudaStream_t alloc_st);
void tma_free_buffers(TmaBuffers *b, cudaStream_t st);
// steps_ps (device, ns ints, or nullptr): per-sample step counts, nsteps = their maximum.
mfmc_status run_solve_tma_core(const Model &m, int kahan, int variant, const StepCoef *coef, const float *u0,
                               size_t ns, int nsteps, const int *steps_ps, float *uT, double *ubar, double *ooi,
                               const TmaBuffers &b, cudaStream_t st);
mfmc_status run_resident_steps(const Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                               const int *steps_ps, float *uT, double *ubar, double *ooi, cudaStream_t st);
// OoI from per-tile partials (tile order), and copying fields into a ghost frame.
mfmc_status launch_finalize(const double *partials, int tiles, size_t ns, int n, double *ubar, double *ooi,
                            cudaStream_t st);
mfmc_status launch_pad(const float *u0, float *padded, int n, int G, size_t ns, cudaStream_t st);
// Warp-strip row-streaming kernel: buffers and solve; bh = rows per work range (0: the batch's
// rows split evenly over the resident warps), rx = columns per thread (4).
mfmc_status rows_alloc_buffers(const Model &m, int bh, size_t ns, TmaBuffers *b, cudaStream_t alloc_st);
mfmc_status run_solve_rows_core(const Model &m, int bh, int rx, const StepCoef *coef, const float *u0, size_t ns,
                                int nsteps, const int *steps_ps, float *uT, double *ubar, double *ooi,
                                const TmaBuffers &b, cudaStream_t st);
mfmc_status run_solve_rows(Model &m, int bh, int rx, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                           float *uT, double *ubar, double *ooi, cudaStream_t st);
bool rows_supported(const Model &m, int rx);
// The TMA pipeline with an explicit tile-shape variant (autotuner).
mfmc_status run_solve_tma(Model &m, int kahan, int variant, const StepCoef *coef, const float *u0, size_t ns,
                          int nsteps, float *uT, double *ubar, double *ooi, cudaStream_t st);
// The own-FFT spectral path (periodic, beta2 = 0): n = 1024 streamed, n = 64 and 128 resident in
// the register-transform form, other even n <= 128 in the resident mixed-radix form.
bool spectral_supported(const Model &m);
mfmc_status run_solve_spectral(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps, float *uT,
                               double *ubar, double *ooi, cudaStream_t st);
// K^(ky, kx) / n^2 of the model's FP32 disc weights (summed in FP64), at [kx][ky].
std::vector<float> spectral_khat(const Model &m, int n);
// Resident spectral solves (spectral_resident.cu): one launch over the (model, sample group) items
// of up to kSrMaxModels models with n <= 128 (register transforms on 64 and 128, mixed-radix
// transforms on other n).
constexpr int kSrMaxModels = 16;
struct SrBatch {
    const float *u0 = nullptr;      // [ns][n][n]
    float *uT = nullptr;            // or nullptr
    double *ubar = nullptr, *ooi = nullptr;
    const StepCoef *coef = nullptr;
    const int *steps_ps = nullptr;  // per-sample step counts (device) or nullptr
    size_t ns = 0;
    int nsteps = 0;
};
bool spectral_resident_supported(const Model &m);
// counter: one device int the launch may use as its ticket counter (zeroed on st first)
mfmc_status run_spectral_queue(Model *const *models, const SrBatch *batches, int nm, int *counter, cudaStream_t st);
mfmc_status run_solve_spectral_resident(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps,
                                        float *uT, double *ubar, double *ooi, cudaStream_t st);
// Per-sample FP64 mean (ubar) and OoI of ns fields of n x n, fixed summation order.
mfmc_status launch_field_ooi(const float *u, size_t ns, int n, double *ubar, double *ooi, cudaStream_t st);
mfmc_status run_solve_fft(Model &m, const StepCoef *coef, const float *u0, size_t ns, int nsteps, float *uT,
                          double *ubar, double *ooi, cudaStream_t st);
// FP64 disc sums S = sum_z w_z u_{i+z} of ns fields by cuFFT: u and S are strided per-sample
// blocks (u_dist, s_dist doubles apart); S may not overlap u.
// The real transform of the disc weights (FP64 weights), divided by n^2, at [ky][n/2 + 1].
std::vector<double> khat64_host(const Model &m, int n);
mfmc_status fft64_disc_sums(Model &m, const double *u, size_t u_dist, double *S, size_t s_dist, size_t ns,
                            cudaStream_t st);
// The beta2 > 0 step (semismooth Newton per step: FP64 fields and residual, FP32 preconditioned
// CG corrections, one CTA per sample); eps_dev: per-sample eps (FP64) or nullptr for the nominal eps.
mfmc_status run_solve_active_set(Model &m, const double *eps_dev, const float *u0, size_t ns, int nsteps,
                                 float *uT, double *ubar, double *ooi, cudaStream_t st);
// Whether an algorithm can run this model.
bool algo_supported(const Model &m, int algo);
// Autotuner: time the candidate algorithms on this model once and cache the winner.
mfmc_status autotune(Model &m, cudaStream_t st);

// FP64 statistics / estimator kernels
mfmc_status launch_pilot_stats(int K, int n, const double *ooi, double *out_dev,
                               cudaStream_t st);
mfmc_status launch_estimate(int K, const double *const *ooi_dev_list_dev,
                            const int64_t *m_dev, const double *alpha_dev, double *est_dev,
                            cudaStream_t st);

// host planner (FP64)
mfmc_status plan_from_stats(int K, const double *mean, const double *sigma,
                            const double *rho, const double *costs, double budget, int policy,
                            const int *explicit_idx, int explicit_len, mfmc_plan_t *out);

}  // namespace mfmc

struct mfmc_model : public mfmc::Model {};
