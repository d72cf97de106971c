// C ABI entry points: models, fields, the solve, and the batch call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "mfmc_internal.h"
#include "tma_step.cuh"

namespace mfmc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

mfmc_status fail(mfmc_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

mfmc_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? MFMC_ENOMEM : MFMC_ECUDA;
}

Model::~Model() {
    cudaFree(bufA);
    cudaFree(bufB);
    cudaFree(partials);
    cudaFree(coef);
    cudaFree(d_wtab);
    cudaFree(eps_tmp);
    cudaFree(seeds_tmp);
    cudaFree(theta_tmp);
    cudaFree(u0buf);
    cudaFree(resbuf);
    cudaFree(padA);
    cudaFree(padB);
    cudaFree(d_status);
    cudaFree(d_wtab64);
    cudaFree(d_khat64);
    cudaFree(d_khat32);
    cudaFree(d_tw32);
    cudaFree(sr_counter);
    cudaFree(d_tw64);
    cudaFree(d_wsq);
    cudaFree(as_buf);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (stream) cudaStreamDestroy(stream);
    fft_release(fft);
    fft64_release(fft64);
    spectral_release(spectral);
    cudaFree(d_as_iters);
}

template <typename T>
static mfmc_status grow(T **p, size_t *cap, size_t want) {
    return grow_buffer(p, cap, want);
}

mfmc_status ensure_scratch(Model &m, size_t ns, size_t partials_per_sample) {
    const size_t nn = (size_t)m.d.n * m.d.n;
    if (m.buf_cap < ns || !m.bufA || !m.bufB) {
        cudaFree(m.bufA);
        cudaFree(m.bufB);
        m.bufA = m.bufB = nullptr;
        m.buf_cap = 0;
        cudaError_t e = cudaMalloc((void **)&m.bufA, ns * nn * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (field scratch)");
        e = cudaMalloc((void **)&m.bufB, ns * nn * sizeof(float));
        if (e != cudaSuccess) {
            cudaFree(m.bufA);
            m.bufA = nullptr;
            return cuda_fail(e, "cudaMalloc (field scratch)");
        }
        m.buf_cap = ns;
    }
    return grow(&m.partials, &m.partials_cap, ns * std::max<size_t>(1, partials_per_sample));
}

double resolve_eps(const Model &m, const mfmc_sample_params *p, uint64_t seed) {
    if (p && p->eps > 0) return p->eps;
    if (m.d.eps_hi > m.d.eps_lo) return m.d.eps_lo + (m.d.eps_hi - m.d.eps_lo) * sm64_unit(seed, 0, 0);
    return m.d.eps;
}

void resolve_theta(const mfmc_sample_params *p, uint64_t seed, double th[12]) {
    if (p && p->has_theta) {
        for (int k = 0; k < 4; ++k) {
            th[k] = p->mu[k];
            th[4 + 2 * k] = p->eta[k][0];
            th[5 + 2 * k] = p->eta[k][1];
        }
        return;
    }
    for (int k = 0; k < 4; ++k) {
        th[k] = 0.9 + 0.1 * sm64_unit(seed, 2, 3u * k);
        th[4 + 2 * k] = -0.025 + 0.05 * sm64_unit(seed, 2, 3u * k + 1u);
        th[5 + 2 * k] = -0.025 + 0.05 * sm64_unit(seed, 2, 3u * k + 2u);
    }
}

static mfmc_status validate_desc(const mfmc_model_desc &d, int *R_out) {
    if (d.n < 8 || d.n % 4 != 0 || d.n > 16384) return fail(MFMC_EINVAL, "n must be a multiple of 4 in [8, 16384] (got %d)", d.n);
    if (!(d.delta > 0)) return fail(MFMC_EINVAL, "delta must be > 0");
    const double Rf = d.delta * d.n;
    const double Rr = std::round(Rf);
    // a non-integer delta/h is allowed; the disc is { z : |z| <= delta/h } and only the
    // generic kernel (plain and direct forms) serves it
    const int R = std::fabs(Rf - Rr) <= 1e-9 * std::max(1.0, Rr) ? (int)Rr : (int)std::floor(Rf);
    if (R < 1 || R > kMaxR) return fail(MFMC_EINVAL, "delta/h = %d outside [1, %d]", R, kMaxR);
    if (2 * R + 1 > d.n) return fail(MFMC_EINVAL, "the horizon disc (2R+1 = %d) must fit in one period n = %d", 2 * R + 1, d.n);
    if (!(d.tau > 0)) return fail(MFMC_EINVAL, "tau must be > 0");
    if (!(d.beta1 > 0)) return fail(MFMC_EINVAL, "beta1 must be > 0");
    if (!(d.beta2 >= 0.0)) return fail(MFMC_EINVAL, "beta2 must be >= 0");
    if (d.beta2 > 0.0 && d.bc != MFMC_BC_PERIODIC)
        return fail(MFMC_EINVAL, "beta2 > 0 (the active-set step) runs on the periodic lattice only");
    if (!(d.eps > 0) && !(d.eps_hi > d.eps_lo && d.eps_lo > 0)) return fail(MFMC_EINVAL, "eps must be > 0");
    if (d.eps_hi > d.eps_lo && !(d.eps_lo > 0)) return fail(MFMC_EINVAL, "eps range must be positive");
    if (!(d.c_F >= 0)) return fail(MFMC_EINVAL, "c_F must be >= 0");
    if (d.nsteps < 0) return fail(MFMC_EINVAL, "nsteps must be >= 0");
    if (d.kernel != MFMC_KERNEL_CONSTANT && d.kernel != MFMC_KERNEL_GAUSSIAN) return fail(MFMC_EINVAL, "unknown kernel");
    if (d.kernel == MFMC_KERNEL_GAUSSIAN && !(d.delta_hf > 0)) return fail(MFMC_EINVAL, "delta_hf must be > 0");
    if (d.bc != MFMC_BC_PERIODIC && d.bc != MFMC_BC_COLLAR) return fail(MFMC_EINVAL, "unknown boundary");
    if (d.bc == MFMC_BC_COLLAR && !(d.bc_value >= -1.0 && d.bc_value <= 1.0))
        return fail(MFMC_EINVAL, "the collar value must lie in [-1, 1]");
    if (d.ic != MFMC_IC_UNIFORM && d.ic != MFMC_IC_SMOOTHED_GAUSS && d.ic != MFMC_IC_NUCLEI) return fail(MFMC_EINVAL, "unknown ic");
    if (!(d.ic_amp >= 0)) return fail(MFMC_EINVAL, "ic_amp must be >= 0");
    if (d.ic_base_n < 0 || (d.ic_base_n > 0 && (d.ic_base_n % d.n != 0 || d.ic_base_n > 16384)))
        return fail(MFMC_EINVAL, "ic_base_n must be 0 or a multiple of n up to 16384");
    if ((int)d.algo < MFMC_ALGO_AUTO || (int)d.algo > MFMC_ALGO_SPECTRAL) return fail(MFMC_EINVAL, "unknown algo");
    *R_out = R;
    return MFMC_OK;
}

}  // namespace mfmc

using namespace mfmc;

extern "C" {

const char *mfmc_version(void) { return "mfmc-nlch 1.0 (sm_103a)"; }

const char *mfmc_last_error(void) { return g_err; }

mfmc_status mfmc_model_create(const mfmc_model_desc *desc, mfmc_model **out) {
    if (!desc || !out) return fail(MFMC_EINVAL, "NULL argument");
    *out = nullptr;
    int R = 0;
    mfmc_status s = validate_desc(*desc, &R);
    if (s != MFMC_OK) return s;
    mfmc_model *m = new (std::nothrow) mfmc_model();
    if (!m) return fail(MFMC_ENOMEM, "host allocation failed");
    m->d = *desc;
    m->R = R;
    {
        const double Rf = desc->delta * desc->n;
        m->integer_R = std::fabs(Rf - R) <= 1e-9 * std::max(1.0, (double)R) ? 1 : 0;
        m->r2max = m->integer_R ? R * R : (int)std::floor(Rf * Rf * (1.0 + 1e-12));
    }
    int count = 0;
    for (int d = 0; d <= R; ++d) {
        int w = 0;
        while ((w + 1) * (w + 1) <= m->r2max - d * d) ++w;
        m->widths[d] = w;
        count += (2 * w + 1) * (d == 0 ? 1 : 2);
    }
    m->disc = count;
    const double h = 1.0 / desc->n;
    if (desc->kernel == MFMC_KERNEL_CONSTANT) {
        // gamma = 8 eps^2 / (pi delta^4): h^2 gamma = eps^2 * ahat, unit weights
        m->ahat = 8.0 * h * h / (M_PI * std::pow(desc->delta, 4));
        m->chat = (double)count;
        m->chat64 = (double)count;
    } else {
        // Gaussian weights / eps^2: h^2 4 / (pi s^4) exp(-r^2 / s^2), s = delta_hf / 3
        const double sg = desc->delta_hf / 3.0;
        const double pref = h * h * 4.0 / (M_PI * std::pow(sg, 4));
        m->ahat = 1.0;
        m->wtab.assign(m->r2max + 1, 0.f);
        std::vector<double> wd(m->r2max + 1, 0.0);
        for (int r2 = 0; r2 <= m->r2max; ++r2) {
            wd[r2] = pref * std::exp(-(double)r2 * h * h / (sg * sg));
            m->wtab[r2] = (float)wd[r2];
        }
        double c = 0.0;
        for (int dy = -R; dy <= R; ++dy) {
            const int w = m->widths[dy < 0 ? -dy : dy];
            for (int dx = -w; dx <= w; ++dx) c += (double)m->wtab[dx * dx + dy * dy];
        }
        m->chat = c;  // sum of the FP32 weights the kernel uses
        m->wtab64 = wd;
        double c64 = 0.0;
        for (int dy = -R; dy <= R; ++dy) {
            const int w = m->widths[dy < 0 ? -dy : dy];
            for (int dx = -w; dx <= w; ++dx) c64 += wd[dx * dx + dy * dy];
        }
        m->chat64 = c64;
    }
    // the weighted TMA form's table: what(|dx|, |dy|) inside the disc, zero outside
    m->wsq.assign((size_t)(R + 1) * (R + 1), 0.f);
    for (int dy = 0; dy <= R; ++dy)
        for (int dx = 0; dx <= m->widths[dy]; ++dx)
            m->wsq[(size_t)dy * (R + 1) + dx] = desc->kernel == MFMC_KERNEL_CONSTANT ? 1.f : m->wtab[dx * dx + dy * dy];
    m->algo = desc->algo;
    m->tuned = 0;
    if (m->algo != MFMC_ALGO_AUTO && !algo_supported(*m, m->algo)) {
        delete m;
        return fail(MFMC_EINVAL, "algorithm %d does not support this model (R=%d, kernel=%d)", (int)desc->algo, R,
                    (int)desc->kernel);
    }
    *out = m;
    return MFMC_OK;
}

void mfmc_model_destroy(mfmc_model *model) { delete model; }

mfmc_status mfmc_model_set_iteration_limits(mfmc_model *m, int newton_max, int cg_max) {
    if (!m) return fail(MFMC_EINVAL, "NULL model");
    if (newton_max < 0 || newton_max > 100000 || cg_max < 0 || cg_max > 100000)
        return fail(MFMC_EINVAL, "iteration limits outside [0, 100000]");
    std::lock_guard<std::mutex> lk(m->mu);
    m->as_newton_max = newton_max > 0 ? newton_max : kAsNewtonMax;
    m->as_cg_max = cg_max > 0 ? cg_max : kAsCgMax;
    return MFMC_OK;
}

mfmc_status mfmc_model_solver_stats(const mfmc_model *m, uint64_t *newton_iters, uint64_t *cg_iters) {
    if (!m) return fail(MFMC_EINVAL, "NULL model");
    unsigned long long it[2] = {0, 0};
    if (m->d_as_iters) MFMC_CUDA(cudaMemcpy(it, m->d_as_iters, sizeof(it), cudaMemcpyDeviceToHost));
    if (newton_iters) *newton_iters = it[0];
    if (cg_iters) *cg_iters = it[1];
    return MFMC_OK;
}

mfmc_status mfmc_model_query(const mfmc_model *m, mfmc_model_info *out) {
    if (!m || !out) return fail(MFMC_EINVAL, "NULL argument");
    out->R = m->R;
    out->disc_points = m->disc;
    out->c_gamma = m->d.eps * m->d.eps * m->ahat * m->chat;
    out->xi = out->c_gamma - m->d.c_F;
    out->algo = m->algo;
    out->field_bytes = (size_t)m->d.n * m->d.n * sizeof(float);
    out->tile_variant = m->tma_variant;
    out->band_height = m->rows_bh;
    out->columns_per_thread = m->rows_rx;
    return MFMC_OK;
}

mfmc_status mfmc_model_set_tile_variant(mfmc_model *m, int variant) {
    if (!m || variant < 0 || variant >= kTmaVariants) return fail(MFMC_EINVAL, "invalid tile variant");
    std::lock_guard<std::mutex> lk(m->mu);
    m->tma_variant = variant;
    return MFMC_OK;
}

mfmc_status mfmc_model_set_band_height(mfmc_model *m, int rows, int columns_per_thread) {
    if (!m || (rows != 0 && (rows < 8 || rows > 16384)) || columns_per_thread != 4)
        return fail(MFMC_EINVAL, "invalid band height or columns per thread");
    std::lock_guard<std::mutex> lk(m->mu);
    m->rows_bh = rows;
    m->rows_rx = columns_per_thread;
    return MFMC_OK;
}

mfmc_status mfmc_sample_eps(const mfmc_model *m, const mfmc_sample_params *params, const uint64_t *seeds,
                            size_t ns, double *eps_out) {
    if (!m || (ns && (!seeds || !eps_out))) return fail(MFMC_EINVAL, "NULL argument");
    for (size_t i = 0; i < ns; ++i) eps_out[i] = resolve_eps(*m, params ? params + i : nullptr, seeds[i]);
    return MFMC_OK;
}

mfmc_status mfmc_init_fields(const mfmc_model *cm, const mfmc_sample_params *params, const uint64_t *seeds,
                             size_t ns, float *u0, void *stream) {
    if (!cm) return fail(MFMC_EINVAL, "NULL model");
    if (ns == 0) return MFMC_OK;
    if (!seeds || !u0) return fail(MFMC_EINVAL, "NULL argument");
    if (ns > (size_t)kMaxNs) return fail(MFMC_EINVAL, "too many samples");
    mfmc_model *m = const_cast<mfmc_model *>(cm);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> theta(12 * ns, 0.0);
    if (m->d.ic == MFMC_IC_NUCLEI)
        for (size_t i = 0; i < ns; ++i) resolve_theta(params ? params + i : nullptr, seeds[i], &theta[12 * i]);
    // the copies below are issued after any earlier use of these buffers on `st`
    if (m->seeds_cap < ns) {
        MFMC_CUDA(cudaStreamSynchronize(st));
        cudaFree(m->seeds_tmp);
        cudaFree(m->theta_tmp);
        m->seeds_tmp = nullptr;
        m->theta_tmp = nullptr;
        m->seeds_cap = 0;
        MFMC_CUDA(cudaMalloc((void **)&m->seeds_tmp, ns * sizeof(uint64_t)));
        MFMC_CUDA(cudaMalloc((void **)&m->theta_tmp, ns * 12 * sizeof(double)));
        m->seeds_cap = ns;
    }
    MFMC_CUDA(cudaMemcpyAsync(m->seeds_tmp, seeds, ns * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    MFMC_CUDA(cudaMemcpyAsync(m->theta_tmp, theta.data(), ns * 12 * sizeof(double), cudaMemcpyHostToDevice, st));
    mfmc_status s = launch_init_fields(*m, m->seeds_tmp, m->theta_tmp, ns, u0, st);
    if (s != MFMC_OK) return s;
    // the host vectors must outlive the copies
    MFMC_CUDA(cudaStreamSynchronize(st));
    return MFMC_OK;
}

static mfmc_status solve_impl(mfmc_model *m, int algo, const double *eps, const float *u0, size_t ns, float *uT,
                              double *ubar, double *ooi, cudaStream_t st, int nsteps = -1) {
    if (nsteps < 0) nsteps = m->d.nsteps;
    if (ns == 0) return MFMC_OK;
    if (!u0) return fail(MFMC_EINVAL, "NULL u0");
    if (uT && uT == u0) return fail(MFMC_EINVAL, "uT must not alias u0");
    if (ns > (size_t)kMaxNs) return fail(MFMC_EINVAL, "too many samples");
    std::lock_guard<std::mutex> lk(m->mu);
    if (algo == MFMC_ALGO_AUTO) {
        if (!m->tuned) {
            mfmc_status s = autotune(*m, st);
            if (s != MFMC_OK) return s;
        }
        algo = m->algo;
    }
    if (!algo_supported(*m, algo)) return fail(MFMC_EINVAL, "algorithm %d does not support this model", algo);
    if (algo == MFMC_ALGO_ACTIVE_SET) return run_solve_active_set(*m, eps, u0, ns, nsteps, uT, ubar, ooi, st);
    mfmc_status s = grow(&m->coef, &m->coef_cap, ns);
    if (s != MFMC_OK) return s;
    if (m->d.kernel == MFMC_KERNEL_GAUSSIAN && !m->d_wtab) {
        MFMC_CUDA(cudaMalloc((void **)&m->d_wtab, m->wtab.size() * sizeof(float)));
        MFMC_CUDA(cudaMemcpy(m->d_wtab, m->wtab.data(), m->wtab.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    // The launch sequence of a solve (coefficients, ~nsteps step kernels, OoI) is replayed as a
    // CUDA graph while the call's key (algorithm, shape, every pointer it touches, stream) is
    // unchanged: the first call with a key runs directly (sizing scratch), then is captured.
    const bool graphable = !m->graphs_off && algo != MFMC_ALGO_RESIDENT && algo != MFMC_ALGO_PLAIN &&
                           algo != MFMC_ALGO_FFT && nsteps > 0;
    auto key = [&]() {
        return std::vector<uintptr_t>{(uintptr_t)algo, (uintptr_t)m->tma_variant, (uintptr_t)m->rows_bh,
                                      (uintptr_t)m->rows_rx, (uintptr_t)ns, (uintptr_t)nsteps, (uintptr_t)eps,
                                      (uintptr_t)u0, (uintptr_t)uT, (uintptr_t)ubar, (uintptr_t)ooi,
                                      (uintptr_t)st, (uintptr_t)m->coef, (uintptr_t)m->bufA, (uintptr_t)m->bufB,
                                      (uintptr_t)m->padA, (uintptr_t)m->padB, (uintptr_t)m->partials,
                                      (uintptr_t)m->map_sw, (uintptr_t)m->map_sh, (uintptr_t)m->d_wtab};
    };
    if (graphable && m->gexec && m->gkey == key()) {
        MFMC_CUDA(cudaGraphLaunch(m->gexec, st));
        return MFMC_OK;
    }
    s = launch_coefficients(*m, eps, ns, m->coef, st);
    if (s != MFMC_OK) return s;
    s = run_solve(*m, algo, m->coef, u0, ns, nsteps, uT, ubar, ooi, st);
    if (s != MFMC_OK || !graphable) return s;
    if (m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        (void)cudaGetLastError();
        m->graphs_off = 1;
        return MFMC_OK;
    }
    mfmc_status cs = launch_coefficients(*m, eps, ns, m->coef, st);
    if (cs == MFMC_OK) cs = run_solve(*m, algo, m->coef, u0, ns, nsteps, uT, ubar, ooi, st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (cs == MFMC_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&m->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cs != MFMC_OK || e != cudaSuccess) {
        (void)cudaGetLastError();
        m->gexec = nullptr;
        m->graphs_off = 1;  // keep launching directly
        set_error("");
        return MFMC_OK;
    }
    m->gkey = key();
    return MFMC_OK;
}

mfmc_status mfmc_solve_fields(const mfmc_model *cm, const double *eps, const float *u0, size_t ns, float *uT,
                              double *ubar, double *ooi, void *stream) {
    if (!cm) return fail(MFMC_EINVAL, "NULL model");
    mfmc_model *m = const_cast<mfmc_model *>(cm);
    return solve_impl(m, m->tuned ? m->algo : (int)m->d.algo, eps, u0, ns, uT, ubar, ooi, (cudaStream_t)stream);
}

mfmc_status mfmc_solve_fields_algo(const mfmc_model *cm, int algo, const double *eps, const float *u0, size_t ns,
                                   float *uT, double *ubar, double *ooi, void *stream) {
    if (!cm) return fail(MFMC_EINVAL, "NULL model");
    if (algo < MFMC_ALGO_AUTO || algo > MFMC_ALGO_SPECTRAL) return fail(MFMC_EINVAL, "unknown algo");
    return solve_impl(const_cast<mfmc_model *>(cm), algo, eps, u0, ns, uT, ubar, ooi, (cudaStream_t)stream);
}

// Batch call: samples grouped by model; each group is solved from fields built on the
// device in the model's own buffers and stream, so groups of different fidelities
// overlap on the GPU.  Results are gathered back in sample order.
mfmc_status mfmc_solve_batch(mfmc_model *const *models, const mfmc_sample_params *params, const uint64_t *seeds,
                             size_t ns, double *ooi_out, double *ubar_out) {
    if (ns == 0) return MFMC_OK;
    if (!models || !seeds || !ooi_out) return fail(MFMC_EINVAL, "NULL argument");
    if (ns > (size_t)kMaxNs) return fail(MFMC_EINVAL, "too many samples");
    // groups of (model, number of steps), in order of first appearance
    typedef std::pair<mfmc_model *, int> Key;
    std::map<Key, std::vector<size_t>> groups;
    std::vector<Key> order;
    for (size_t i = 0; i < ns; ++i) {
        if (!models[i]) return fail(MFMC_EINVAL, "NULL model at sample %zu", i);
        const int k = (params && params[i].nsteps > 0) ? params[i].nsteps : models[i]->d.nsteps;
        const Key key(models[i], k);
        auto it = groups.find(key);
        if (it == groups.end()) order.push_back(key);
        groups[key].push_back(i);
    }
    // groups of one model run one after the other on that model's stream and buffers
    std::vector<std::vector<double>> host_res(order.size());
    for (size_t g = 0; g < order.size(); ++g) {
        mfmc_model *m = order[g].first;
        const int gsteps = order[g].second;
        const std::vector<size_t> &idx = groups[order[g]];
        const size_t k = idx.size();
        const size_t nn = (size_t)m->d.n * m->d.n;
        {
            std::lock_guard<std::mutex> lk(m->mu);
            if (!m->stream) MFMC_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
            MFMC_CUDA(cudaStreamSynchronize(m->stream));
            // a flag left by an earlier solve whose results nobody waited for is not this call's
            if (m->d_status) MFMC_CUDA(cudaMemset(m->d_status, 0, sizeof(int)));
            mfmc_status s = grow_buffer(&m->u0buf, &m->u0_cap, k * nn);
            if (s == MFMC_OK) s = grow_buffer(&m->eps_tmp, &m->eps_cap, k);
            if (s == MFMC_OK) s = grow_buffer(&m->resbuf, &m->res_cap, 2 * k);
            if (s != MFMC_OK) return s;
        }
        std::vector<uint64_t> sd(k);
        std::vector<mfmc_sample_params> pp(params ? k : 0);
        std::vector<double> ep(k);
        for (size_t q = 0; q < k; ++q) {
            sd[q] = seeds[idx[q]];
            if (params) pp[q] = params[idx[q]];
            ep[q] = resolve_eps(*m, params ? &params[idx[q]] : nullptr, sd[q]);
        }
        MFMC_CUDA(cudaMemcpyAsync(m->eps_tmp, ep.data(), k * sizeof(double), cudaMemcpyHostToDevice, m->stream));
        mfmc_status s = mfmc_init_fields(m, params ? pp.data() : nullptr, sd.data(), k, m->u0buf, m->stream);
        if (s != MFMC_OK) return s;
        s = solve_impl(m, m->tuned ? m->algo : (int)m->d.algo, m->eps_tmp, m->u0buf, k, nullptr, m->resbuf + k,
                       m->resbuf, m->stream, gsteps);
        if (s != MFMC_OK) return s;
        host_res[g].resize(2 * k);
        MFMC_CUDA(cudaMemcpyAsync(host_res[g].data(), m->resbuf, 2 * k * sizeof(double), cudaMemcpyDeviceToHost,
                                  m->stream));
        // the next group of the same model reuses its buffers
        bool again = false;
        for (size_t h = g + 1; h < order.size(); ++h) again |= order[h].first == m;
        if (again) MFMC_CUDA(cudaStreamSynchronize(m->stream));
    }
    for (size_t g = 0; g < order.size(); ++g) {
        mfmc_model *m = order[g].first;
        MFMC_CUDA(cudaStreamSynchronize(m->stream));
        if (m->d_status) {
            int flag = 0;
            MFMC_CUDA(cudaMemcpy(&flag, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
            if (flag) {
                // reported once: the next call starts with the flag cleared
                MFMC_CUDA(cudaMemset(m->d_status, 0, sizeof(int)));
                return fail(MFMC_ETIMEOUT, "a device-side wait or an iteration bound gave up");
            }
        }
        const std::vector<size_t> &idx = groups[order[g]];
        const size_t k = idx.size();
        for (size_t q = 0; q < k; ++q) {
            ooi_out[idx[q]] = host_res[g][q];
            if (ubar_out) ubar_out[idx[q]] = host_res[g][k + q];
        }
    }
    return MFMC_OK;
}

}  // extern "C"
