// Host side of the per-work-item trace (trace.cuh): one ring per device, turned on by
// mfmc_trace_enable or, at a device's first traced launch, by the environment variable
// MFMC_TRACE=<records>.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>
#include <vector>

#include "mfmc_internal.h"
#include "trace.cuh"

namespace mfmc {

struct TraceState {
    TraceBuf buf;
    bool env_checked = false;
};

static std::mutex g_trace_mu;
static std::vector<TraceState> g_trace;  // per device

static mfmc_status trace_set(int dev, size_t capacity) {
    TraceState &s = g_trace[dev];
    s.env_checked = true;
    if (s.buf.rec) {
        MFMC_CUDA(cudaDeviceSynchronize());  // no launch still writes the old ring
        cudaFree(s.buf.rec);
        cudaFree(s.buf.count);
    }
    s.buf = TraceBuf();
    if (capacity == 0) return MFMC_OK;
    MFMC_CUDA(cudaMalloc((void **)&s.buf.rec, capacity * sizeof(TraceRec)));
    MFMC_CUDA(cudaMalloc((void **)&s.buf.count, sizeof(unsigned long long)));
    MFMC_CUDA(cudaMemset(s.buf.count, 0, sizeof(unsigned long long)));
    s.buf.cap = capacity;
    return MFMC_OK;
}

TraceBuf trace_buf() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TraceBuf();
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if ((int)g_trace.size() <= dev) g_trace.resize(dev + 1);
    TraceState &s = g_trace[dev];
    if (!s.env_checked) {
        s.env_checked = true;
        const char *e = std::getenv("MFMC_TRACE");
        const long long cap = e ? std::atoll(e) : 0;
        if (cap > 0 && cap <= (1ll << 28) && trace_set(dev, (size_t)cap) != MFMC_OK) s.buf = TraceBuf();
    }
    return s.buf;
}

}  // namespace mfmc

using namespace mfmc;

extern "C" mfmc_status mfmc_trace_enable(size_t capacity) {
    if (capacity > ((size_t)1 << 28)) return fail(MFMC_EINVAL, "trace capacity above 2^28 records");
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if ((int)g_trace.size() <= dev) g_trace.resize(dev + 1);
    return trace_set(dev, capacity);
}

extern "C" mfmc_status mfmc_trace_read(mfmc_trace_record *out, size_t max, size_t *n_out, uint64_t *dropped_out) {
    if (n_out) *n_out = 0;
    if (dropped_out) *dropped_out = 0;
    if (max > 0 && !out) return fail(MFMC_EINVAL, "NULL output with max > 0");
    int dev = 0;
    MFMC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if ((int)g_trace.size() <= dev || !g_trace[dev].buf.rec) return fail(MFMC_EINVAL, "tracing is off on this device");
    const TraceBuf &b = g_trace[dev].buf;
    MFMC_CUDA(cudaDeviceSynchronize());  // every traced launch has written its records
    unsigned long long count = 0;
    MFMC_CUDA(cudaMemcpy(&count, b.count, sizeof(count), cudaMemcpyDeviceToHost));
    const unsigned long long held = count < b.cap ? count : b.cap;
    std::vector<TraceRec> ring(held);
    if (held) MFMC_CUDA(cudaMemcpy(ring.data(), b.rec, held * sizeof(TraceRec), cudaMemcpyDeviceToHost));
    // oldest first: after a wrap the oldest held record sits at count mod cap
    const unsigned long long first = count > b.cap ? count % b.cap : 0;
    const size_t n = (size_t)(held < max ? held : max);
    for (size_t i = 0; i < n; ++i) {
        const TraceRec &r = ring[(first + i) % (held ? held : 1)];
        out[i].t0_ns = r.t0;
        out[i].t1_ns = r.t1;
        out[i].item = r.item;
        out[i].sm = r.sm;
        out[i].kind = r.kind;
        out[i].step = r.step;
    }
    if (n_out) *n_out = n;
    if (dropped_out) *dropped_out = count - n;
    MFMC_CUDA(cudaMemset(b.count, 0, sizeof(unsigned long long)));
    return MFMC_OK;
}
