// The resident spectral queue: one launch over the (model, sample group) items of up to
// kSrMaxModels periodic beta2 = 0 models with n <= 128, each item a whole solve on chip.
//
// Items of a model on n = 128 (one sample) or n = 64 (four samples) run the register-transform
// solve of spectral.cu (small_solve); items of any other n run the mixed-radix solve of
// smem_fft.cuh (one sample; the paper's n = 88 on its compile-time plan).  The CTA has the
// register form's nine warps, and its shared memory is the largest any of the launch's models
// needs; a launch without register-form items uses a form of the kernel that fits two CTAs per
// SM.  Kernel and launcher in spectral.cu, host set-up in spectral_resident.cu.
#pragma once

#include "mfmc_internal.h"
#include "smem_fft.cuh"
#include "trace.cuh"

namespace mfmc {

enum : int { kSqGeneric = 0, kSqSmall64 = 2, kSqSmall128 = 4 };  // item kinds (register form: E)
constexpr int kSqThreads = 288;                                    // nine warps

struct SqModelDev {
    const float *u0;       // [ns][n][n] initial fields
    float *uT;             // final fields, or nullptr
    double *ubar, *ooi;    // per sample, or nullptr
    const StepCoef *coef;  // per sample
    const int *steps_ps;   // per-sample step counts, or nullptr: nsteps for every sample
    const float *khat;     // K^(ky, kx) / n^2: [ky][n/2 + 1] (mixed-radix), [kx][ky] (register form)
    const float2 *tw;      // W_n^j, j < n (mixed-radix); W_n^(n1 k2) at [n1][k2], 33 per n1 (register)
    FftPlan plan;
    int kind;              // kSqGeneric, kSqSmall64 or kSqSmall128
    int spc;               // samples per item
    int ns, nsteps;
};

struct SqArgs {
    SqModelDev m[kSrMaxModels];
    int begin[kSrMaxModels + 1];  // items of model k: [begin[k], begin[k + 1])
    int nm, total;
    int *counter;                 // zero at launch
    TraceBuf trace;
};

// Dynamic shared memory of one item kind on an n x n lattice.
size_t spectral_queue_smem(int kind, int n);
// The register form's tables of a model with n = 64 or 128 (made once per model and device; the
// register transforms' constants are written on the device first).
mfmc_status spectral_small_tables(Model &m, const float **khatT, const float2 **tw);
// CTAs of the queue kernel that fit on one SM with `smem` bytes of dynamic shared memory; small:
// the launch has register-form items (the kernel form that carries them).
int spectral_queue_blocks_per_sm(bool small, size_t smem);
mfmc_status launch_spectral_queue(bool small, const SqArgs &a, int grid, size_t smem, cudaStream_t st);

}  // namespace mfmc
