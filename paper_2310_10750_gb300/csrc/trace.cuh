// Per-work-item trace of the queue kernels (MFMC_TRACE; mfmc_trace_enable / mfmc_trace_read).
//
// When tracing is on for a device, the kernels that take work items from a queue (the resident
// spectral queue, the mixed-fidelity step queue) and the beta2 > 0 solver (one item per sample)
// append one record per item to a ring in device memory: the global timer at the item's start
// and end, the item's index, the SM that ran it, the kernel and the time step.  A record's slot
// is taken with one atomic add on the ring's counter; when more records arrive than the ring
// holds, the newest overwrite the oldest.  Off (rec == nullptr), a kernel only tests a pointer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mfmc {

enum : uint32_t { kTraceSpectralQueue = 1, kTraceMixedStep = 2, kTraceActiveSet = 3 };

struct TraceRec {
    unsigned long long t0, t1;  // global timer (ns) at the item's start and end
    uint32_t item, sm, kind, step;
};

struct TraceBuf {
    TraceRec *rec = nullptr;             // the ring, or nullptr: tracing off
    unsigned long long *count = nullptr; // records written since the last read
    unsigned long long cap = 0;
};

// The calling thread's current device's ring (off unless mfmc_trace_enable or the MFMC_TRACE
// environment variable turned it on there).
TraceBuf trace_buf();

__device__ __forceinline__ unsigned long long trace_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One record (called by one thread per item).
__device__ __forceinline__ void trace_put(const TraceBuf &tb, uint32_t kind, uint32_t item, uint32_t step,
                                          unsigned long long t0) {
    if (!tb.rec) return;
    uint32_t sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    const unsigned long long i = atomicAdd(tb.count, 1ull);
    TraceRec r;
    r.t0 = t0;
    r.t1 = trace_clock();
    r.item = item;
    r.sm = sm;
    r.kind = kind;
    r.step = step;
    tb.rec[i % tb.cap] = r;
}

}  // namespace mfmc
