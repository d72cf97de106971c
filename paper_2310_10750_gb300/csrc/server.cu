// Continuous-batching request loop (serving).
//
// Requests (model, seed, optional parameters, per-request step count) are queued by
// mfmc_submit.  A loop thread admits queued requests in arrival order while fewer than
// max_slots are in flight and their device memory fits the budget; the requests of one
// model admitted together form a cohort.  Each cohort runs its whole solve (initial
// fields, steps, OoI) asynchronously on a stream of its own, so cohorts admitted while
// others are on the GPU run alongside them.  Samples of a cohort may have different step
// counts: the kernels skip a sample once its own steps are done.  When a cohort's
// completion event fires, its results are posted, its memory and slots are released and
// further requests are admitted.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mfmc_internal.h"

namespace mfmc {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerReq {
    uint64_t ticket;
    mfmc_model *model;
    mfmc_sample_params p;
    int has_p;
    uint64_t seed;
    int nsteps;
    double t_submit;
    double t_admit = -1.0;
};

struct Cohort {
    mfmc_model *model = nullptr;
    std::vector<ServerReq> reqs;
    std::vector<int> slots;  // result slot of each request
    size_t bytes = 0;
    bool resident = false;
    bool rows = false;       // the model was tuned to the row-streaming kernel
    int variant = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    float *u0 = nullptr;
    StepCoef *coef = nullptr;
    double *eps = nullptr, *out = nullptr, *theta = nullptr;
    uint64_t *seeds = nullptr;
    int *steps = nullptr, *slot_dev = nullptr;
    TmaBuffers tb;
};

// Results go straight to mapped pinned host memory: res[2 * slot] = OoI, res[2 * slot + 1] =
// mean, written by the device once the cohort's solve is done.
__global__ void scatter_results_kernel(const double *out, const int *slots, int k, double *res) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    res[2 * slots[q]] = out[q];
    res[2 * slots[q] + 1] = out[k + q];
}

// Device bytes one request holds while admitted.
static size_t request_bytes(const Model &m, bool resident) {
    const size_t nn = (size_t)m.d.n * m.d.n;
    size_t b = nn * sizeof(float) + 256;  // initial field + small per-sample arrays
    if (!resident) {
        const size_t G = (m.R + 3) & ~3, P = m.d.n + 2 * G;
        int tiles_x = 0;
        b += 2 * P * P * sizeof(float) + (size_t)tma_tiles(m, m.tma_variant, &tiles_x) * sizeof(double);
    }
    return b;
}

static bool use_resident(const Model &m) { return algo_supported(m, MFMC_ALGO_RESIDENT); }

}  // namespace mfmc

using namespace mfmc;

struct mfmc_server {
    size_t budget = 0;
    int max_slots = 0;
    int device = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServerReq> pending;
    std::vector<Cohort *> running;
    std::unordered_map<uint64_t, std::pair<double, double>> results;
    // submit, admit and completion times of every finished request (kept until destroy)
    std::unordered_map<uint64_t, std::array<double, 3>> times;
    double t0 = 0;  // server creation
    std::unordered_set<uint64_t> open;  // submitted, result not yet polled
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0, peak_bytes = 0;
    int inflight = 0, peak_inflight = 0;
    bool stop = false;
    mfmc_status error = MFMC_OK;
    char err[256] = "";
    std::vector<double> latencies;
    uint64_t submitted = 0, completed = 0, rejected = 0;
    double t_first = -1, t_last = -1;
    double *res_host = nullptr, *res_dev = nullptr;  // mapped pinned results, 2 per slot
    std::vector<int> free_slots;
};

namespace mfmc {

// Release a cohort's device memory in stream order (no device-wide synchronisation).
static void free_cohort(Cohort *c) {
    if (c->st) {
        for (void *p : {(void *)c->u0, (void *)c->coef, (void *)c->eps, (void *)c->out, (void *)c->theta,
                        (void *)c->seeds, (void *)c->steps, (void *)c->slot_dev})
            if (p) cudaFreeAsync(p, c->st);
        tma_free_buffers(&c->tb, c->st);
        cudaStreamDestroy(c->st);
    }
    if (c->done) cudaEventDestroy(c->done);
    delete c;
}

// Queue one cohort's whole solve on its own stream.
static mfmc_status launch_cohort(Cohort *c, double *res_dev) {
    Model &m = *c->model;
    const size_t k = c->reqs.size();
    const size_t nn = (size_t)m.d.n * m.d.n;
    MFMC_CUDA(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    MFMC_CUDA(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
    cudaStream_t st = c->st;
    MFMC_CUDA(cudaMallocAsync((void **)&c->u0, k * nn * sizeof(float), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->coef, k * sizeof(StepCoef), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->eps, k * sizeof(double), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->out, 2 * k * sizeof(double), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->theta, 12 * k * sizeof(double), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->seeds, k * sizeof(uint64_t), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->steps, k * sizeof(int), st));
    MFMC_CUDA(cudaMallocAsync((void **)&c->slot_dev, k * sizeof(int), st));
    std::vector<uint64_t> seeds(k);
    std::vector<double> eps(k), theta(12 * k, 0.0);
    std::vector<int> steps(k);
    int max_steps = 0;
    for (size_t q = 0; q < k; ++q) {
        const ServerReq &r = c->reqs[q];
        const mfmc_sample_params *p = r.has_p ? &r.p : nullptr;
        seeds[q] = r.seed;
        eps[q] = resolve_eps(m, p, r.seed);
        resolve_theta(p, r.seed, &theta[12 * q]);
        steps[q] = r.nsteps;
        max_steps = std::max(max_steps, r.nsteps);
    }
    MFMC_CUDA(cudaMemcpyAsync(c->seeds, seeds.data(), k * sizeof(uint64_t), cudaMemcpyHostToDevice, c->st));
    MFMC_CUDA(cudaMemcpyAsync(c->eps, eps.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->st));
    MFMC_CUDA(cudaMemcpyAsync(c->theta, theta.data(), 12 * k * sizeof(double), cudaMemcpyHostToDevice, c->st));
    MFMC_CUDA(cudaMemcpyAsync(c->steps, steps.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->st));
    MFMC_CUDA(cudaMemcpyAsync(c->slot_dev, c->slots.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->st));
    mfmc_status s = launch_init_fields(m, c->seeds, c->theta, k, c->u0, c->st);
    if (s == MFMC_OK) s = launch_coefficients(m, c->eps, k, c->coef, c->st);
    if (s != MFMC_OK) return s;
    if (c->resident) {
        s = run_resident_steps(m, c->coef, c->u0, k, max_steps, c->steps, nullptr, c->out + k, c->out, c->st);
    } else if (c->rows) {
        s = rows_alloc_buffers(m, m.rows_bh, k, &c->tb, c->st);
        if (s == MFMC_OK)
            s = run_solve_rows_core(m, m.rows_bh, m.rows_rx, c->coef, c->u0, k, max_steps, c->steps, nullptr,
                                    c->out + k, c->out, c->tb, c->st);
    } else {
        s = tma_alloc_buffers(m, c->variant, k, &c->tb, c->st);
        if (s == MFMC_OK)
            s = run_solve_tma_core(m, 0, c->variant, c->coef, c->u0, k, max_steps, c->steps, nullptr, c->out + k,
                                   c->out, c->tb, c->st);
    }
    if (s != MFMC_OK) return s;
    scatter_results_kernel<<<(unsigned)((k + 127) / 128), 128, 0, c->st>>>(c->out, c->slot_dev, (int)k, res_dev);
    MFMC_LAUNCHED("server launch 1");
    // the host vectors above are pageable: each copy was staged before its call returned
    MFMC_CUDA(cudaEventRecord(c->done, c->st));
    return MFMC_OK;
}

static void server_loop(mfmc_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Cohort *> fresh;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait_for(lk, std::chrono::microseconds(200),
                           [&] { return S->stop || !S->pending.empty() || !S->running.empty(); });
            if (S->stop && S->running.empty()) break;
            // admission in arrival order while slots and memory allow
            std::map<mfmc_model *, Cohort *> by_model;
            while (!S->stop && !S->pending.empty()) {
                ServerReq &r = S->pending.front();
                const bool res = use_resident(*r.model);
                const size_t need = request_bytes(*r.model, res);
                if (S->inflight + 1 > S->max_slots || S->bytes_in_use + need > S->budget) break;
                Cohort *&c = by_model[r.model];
                if (!c) {
                    c = new Cohort();
                    c->model = r.model;
                    c->resident = res;
                    c->rows = !res && r.model->tuned && r.model->algo == MFMC_ALGO_ROWS &&
                              rows_supported(*r.model, r.model->rows_rx);
                    c->variant = r.model->tma_variant;
                    fresh.push_back(c);
                }
                r.t_admit = now_s();
                c->reqs.push_back(r);
                c->slots.push_back(S->free_slots.back());
                S->free_slots.pop_back();
                c->bytes += need;
                S->bytes_in_use += need;
                S->inflight += 1;
                S->pending.pop_front();
            }
            S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
            S->peak_inflight = std::max(S->peak_inflight, S->inflight);
        }
        for (Cohort *c : fresh) {
            mfmc_status s = launch_cohort(c, S->res_dev);
            std::lock_guard<std::mutex> lk(S->mu);
            if (s != MFMC_OK) {
                S->error = s;
                snprintf(S->err, sizeof(S->err), "%s", mfmc_last_error());
                for (auto &r : c->reqs) {
                    S->results[r.ticket] = {-1.0, -1.0};
                    S->rejected++;
                }
                for (int sl : c->slots) S->free_slots.push_back(sl);
                S->bytes_in_use -= c->bytes;
                S->inflight -= (int)c->reqs.size();
                free_cohort(c);
                continue;
            }
            S->running.push_back(c);
        }
        // completions
        std::vector<Cohort *> finished;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t i = 0; i < S->running.size();) {
                Cohort *c = S->running[i];
                if (cudaEventQuery(c->done) == cudaSuccess) {
                    finished.push_back(c);
                    S->running[i] = S->running.back();
                    S->running.pop_back();
                } else {
                    ++i;
                }
            }
        }
        if (finished.empty()) continue;
        const double t = now_s();
        std::vector<Cohort *> release;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Cohort *c : finished) {
                const size_t k = c->reqs.size();
                for (size_t q = 0; q < k; ++q) {
                    const ServerReq &r = c->reqs[q];
                    const double lat = t - r.t_submit;
                    S->results[r.ticket] = {S->res_host[2 * c->slots[q]], lat};
                    S->times[r.ticket] = {r.t_submit - S->t0, r.t_admit - S->t0, t - S->t0};
                    S->free_slots.push_back(c->slots[q]);
                    S->latencies.push_back(lat);
                    S->completed++;
                }
                S->t_last = t;
                S->bytes_in_use -= c->bytes;
                S->inflight -= (int)k;
                release.push_back(c);
            }
        }
        for (Cohort *c : release) free_cohort(c);
        S->cv.notify_all();
    }
    // drop what was never admitted
    std::lock_guard<std::mutex> lk(S->mu);
    S->pending.clear();
    S->cv.notify_all();
}

}  // namespace mfmc

extern "C" {

mfmc_status mfmc_server_create(size_t hbm_budget_bytes, int max_slots, mfmc_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_slots < 1) return fail(MFMC_EINVAL, "invalid server arguments");
    mfmc_server *S = new (std::nothrow) mfmc_server();
    if (!S) return fail(MFMC_ENOMEM, "host allocation failed");
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->t0 = now_s();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&S->res_host, 2 * (size_t)max_slots * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&S->res_dev, S->res_host, 0);
    if (e != cudaSuccess) {
        if (S->res_host) cudaFreeHost(S->res_host);
        delete S;
        return cuda_fail(e, "server setup");
    }
    for (int i = max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->th = std::thread(server_loop, S);
    *out = S;
    return MFMC_OK;
}

mfmc_status mfmc_submit(mfmc_server *S, const mfmc_model *model, const mfmc_sample_params *params, uint64_t seed,
                        uint64_t *ticket) {
    if (!S || !model || !ticket) return fail(MFMC_EINVAL, "NULL argument");
    mfmc_model *m = const_cast<mfmc_model *>(model);
    if (m->d.kernel != MFMC_KERNEL_CONSTANT || (!use_resident(*m) && !algo_supported(*m, MFMC_ALGO_PREFIX_TMA)))
        return fail(MFMC_EINVAL, "the server runs constant-kernel models with a resident or TMA kernel");
    const int nsteps = (params && params->nsteps > 0) ? params->nsteps : m->d.nsteps;
    if (nsteps < 1) return fail(MFMC_EINVAL, "a served request needs at least one step");
    if (request_bytes(*m, use_resident(*m)) > S->budget)
        return fail(MFMC_EINVAL, "request larger than the server's memory budget");
    ServerReq r;
    r.model = m;
    r.has_p = params != nullptr;
    if (params) r.p = *params;
    r.seed = seed;
    r.nsteps = nsteps;
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(MFMC_EINVAL, "server is stopping");
        r.ticket = S->next_ticket++;
        S->pending.push_back(r);
        S->open.insert(r.ticket);
        S->submitted++;
        if (S->t_first < 0) S->t_first = r.t_submit;
    }
    S->cv.notify_all();
    *ticket = r.ticket;
    return MFMC_OK;
}

mfmc_status mfmc_request_times(mfmc_server *S, uint64_t ticket, double *submit_s, double *admit_s, double *done_s) {
    if (!S) return fail(MFMC_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->times.find(ticket);
    if (it == S->times.end()) {
        if (S->open.count(ticket)) return MFMC_EBUSY;
        return fail(MFMC_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    }
    if (submit_s) *submit_s = it->second[0];
    if (admit_s) *admit_s = it->second[1];
    if (done_s) *done_s = it->second[2];
    return MFMC_OK;
}

mfmc_status mfmc_poll(mfmc_server *S, uint64_t ticket, double *ooi, double *latency_s) {
    if (!S) return fail(MFMC_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
        if (S->open.count(ticket)) return MFMC_EBUSY;
        return fail(MFMC_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    }
    if (it->second.second < 0) {
        S->results.erase(it);
        S->open.erase(ticket);
        return fail(S->error, "request failed: %s", S->err);
    }
    if (ooi) *ooi = it->second.first;
    if (latency_s) *latency_s = it->second.second;
    S->results.erase(it);
    S->open.erase(ticket);
    return MFMC_OK;
}

mfmc_status mfmc_server_drain(mfmc_server *S) {
    if (!S) return fail(MFMC_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait(lk, [&] { return (S->pending.empty() && S->running.empty() && S->inflight == 0) || S->stop; });
    return S->error == MFMC_OK ? MFMC_OK : fail(S->error, "%s", S->err);
}

mfmc_status mfmc_server_get_stats(mfmc_server *S, mfmc_server_stats *out) {
    if (!S || !out) return fail(MFMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
        if (l.empty()) return 0.0;
        size_t i = (size_t)std::ceil(q * l.size()) - 1;
        return l[std::min(i, l.size() - 1)];
    };
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->p50_latency_s = pct(0.50);
    out->p99_latency_s = pct(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_latency_s = l.empty() ? 0.0 : sum / l.size();
    out->samples_per_s = (S->t_last > S->t_first && S->completed) ? S->completed / (S->t_last - S->t_first) : 0.0;
    out->peak_bytes = S->peak_bytes;
    out->peak_inflight = S->peak_inflight;
    return MFMC_OK;
}

void mfmc_server_destroy(mfmc_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaDeviceSynchronize();
    cudaFreeHost(S->res_host);
    delete S;
}

}  // extern "C"
