// Host-side internals shared by the C-ABI translation units (api.cu,
// batch.cu): the context object and the argument/error helpers.
#pragma once

#include "plk_internal.cuh"

struct plk_ctx {
    int device;
    cudaStream_t stream;
    unsigned long long *work;  // work area of the FP64 re-solve (plk::kEmiWorkBytes)
    char err[512];
    plk::Prof prof;
    // aggregated by plk_profile_collect
    int n_agg;
    const char *agg_name[32];
    double agg_ms[32];
    int agg_count[32];
    // launch schedules chosen by the batch autotuner, keyed by (N, window)
    struct Tuned {
        int N, wy, wx, sy, sx;
        plk::Schedule sch;
    } tuned[64];
    int n_tuned;
};

namespace plkapi {

plk_status fail(plk_ctx *ctx, plk_status st, const char *fmt, ...);
plk_status cuda_fail(plk_ctx *ctx, cudaError_t e, const char *what);
bool window_ok(plk_window w);
inline bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }
// The checks every entry point applies to plk_params, and the kernel
// parameters they resolve to (work: the work area of the re-solve).
bool params_ok(const plk_params &p);
void emi_params(const plk_params &p, unsigned long long *work, plk::EmiParams *out);
// plk_params (NULL = defaults) -> kernel parameters, GLRT size and coherence precision.
plk_status resolve_params(plk_ctx *ctx, const plk_params *params, plk::EmiParams *out, double *alpha,
                          int *cov_precision = nullptr, int *ref_scheme = nullptr, float *ps_da_max = nullptr,
                          float *decay = nullptr);

// Make a device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace plkapi
