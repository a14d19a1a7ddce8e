// C ABI of libplk (include/plk.h): argument checking, context and state
// ownership, and the launch sequence of each call.  Host code only.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "api_internal.h"

struct plk_state {
    int device;
    int H, W;
    plk_window win;
    int K_max, M_max;
    int K_used, n_eff, steps, head;
    double W1, W2;       // sums of the merged image weights and of their squares (n_eff, n_eff at equal weights)
    float2 **ring;       // K_max planes [H][W]
    float *sum_pow;      // [H][W]
    float *sum_amp;      // [H][W]
    float *da;           // [H][W] amplitude dispersion of the last step with PS selection
    float *amp_new;      // [H][W] that step's sum of |z| over its real SLCs, at its PS pixels
    uint64_t *mask;      // [Ho][Wo][nwords]
    uint16_t *count;     // [Ho][Wo]
    float2 *C;           // [Ho*Wo][ntri(K_max+M_max)]
    float *phase_all;    // [K_max+M_max][Ho][Wo]
    // plk_ministack_step_host: two device staging buffers for the new SLCs
    // (a step's copy overlaps the previous step's compute), the device outputs,
    // a copy stream and the events ordering them.  Made by the first call.
    struct HostIO {
        bool ready;
        int next;                  // staging buffer of the next call
        float2 *stage[2];          // [M_max][H][W] each
        float *phase;              // [M_max][Ho][Wo]
        float *tcoh;               // [Ho][Wo]
        uint8_t *status;           // [Ho][Wo]
        uint16_t *count;           // [Ho][Wo]
        cudaStream_t copy;
        cudaEvent_t copied[2];     // stage[b] holds the call's SLCs
        cudaEvent_t released[2];   // the last step reading stage[b] has run
        // complex 16-bit input (plk_state_enable_host_io_ci16): the samples
        // land in stage16[b] and are widened into stage[b] on the compute stream
        bool ready16;
        int16_t *stage16[2];       // [M_max][H][W][2] each
        cudaEvent_t widened[2];    // stage16[b] has been widened (free for the next copy)
    } io;
};

namespace {
thread_local char g_noctx_err[512];
}  // namespace

namespace plkapi {

plk_status fail(plk_ctx *ctx, plk_status st, const char *fmt, ...) {
    char *dst = ctx ? ctx->err : g_noctx_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

plk_status cuda_fail(plk_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, PLK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool window_ok(plk_window w) {
    return w.wy >= 1 && w.wx >= 1 && (w.wy & 1) && (w.wx & 1) && w.sy >= 1 && w.sx >= 1 &&
           (long long)w.wy * w.wx <= PLK_MAX_WINDOW;
}

}  // namespace plkapi

using namespace plkapi;

namespace {

// Regularised incomplete beta I_x(a, b) by the continued fraction for the
// incomplete beta function (evaluated with the modified Lentz method), with
// the prefactor x^a (1-x)^b / (a B(a, b)) from log-gamma.  Used for x below
// the mean a/(a+b) only (the GLRT solves in x <= 1/2 with a = b).
double inc_beta_cf(double a, double b, double x) {
    if (x <= 0.0) return 0.0;
    const double lbeta = lgamma(a) + lgamma(b) - lgamma(a + b);
    const double front = exp(a * log(x) + b * log1p(-x) - lbeta) / a;
    const double tiny = 1e-300;
    double f = 1.0, c = 1.0, d = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        const int m = i / 2;
        double num;
        if (i == 0) num = 1.0;
        else if (i % 2 == 0) num = (m * (b - m) * x) / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
        else num = -((a + m) * (a + b + m) * x) / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
        d = 1.0 + num * d;
        if (fabs(d) < tiny) d = tiny;
        d = 1.0 / d;
        c = 1.0 + num / c;
        if (fabs(c) < tiny) c = tiny;
        const double cd = c * d;
        f *= cd;
        if (fabs(1.0 - cd) < 1e-16) break;
    }
    return front * (f - 1.0);
}

}  // namespace

namespace plk {

std::atomic<long long> g_device_allocations{0};

cudaError_t dev_malloc(void **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_device_allocations.fetch_add(1, std::memory_order_relaxed);
    return e;
}

void set_noctx_error(const char *msg) {
    strncpy(g_noctx_err, msg, sizeof(g_noctx_err) - 1);
    g_noctx_err[sizeof(g_noctx_err) - 1] = 0;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cache[dev] = v;
    }
    return cache[dev];
}

}  // namespace plk

using plk::Geom;
using plk::Planes;

bool plkapi::params_ok(const plk_params &p) {
    return (p.alpha > 0 && p.alpha < 1) && (p.beta >= 0 && p.beta < 1) && (p.mu >= 0 && p.mu < 1e6) &&
           (p.tol > 0) && p.max_iter >= 1 && p.max_iter <= 100000 && (p.cond_max > 0) && (p.err_max > 0) &&
           (p.cov_precision == PLK_COV_FP32 || p.cov_precision == PLK_COV_BF16 || p.cov_precision == PLK_COV_FP16) &&
           (p.ref_scheme == PLK_REF_FIRST || p.ref_scheme == PLK_REF_LAST_REAL) &&
           (p.ps_da_max >= 0.f && p.ps_da_max < 1e30f) && (p.decay > 0.f && p.decay <= 1.f);
}

void plkapi::emi_params(const plk_params &p, unsigned long long *work, plk::EmiParams *out) {
    out->work = work;
    out->beta = p.beta;
    out->mu = p.mu;
    out->tol = p.tol;
    out->cond_max = p.cond_max;
    out->err_max = p.err_max;
    out->max_iter = p.max_iter;
    out->fp64_resolve = p.fp64_resolve ? 1 : 0;
}

plk_status plkapi::resolve_params(plk_ctx *ctx, const plk_params *params, plk::EmiParams *out, double *alpha,
                                  int *cov_precision, int *ref_scheme, float *ps_da_max, float *decay) {
    plk_params p;
    if (params) p = *params;
    else plk_default_params(&p);
    if (!params_ok(p)) return fail(ctx, PLK_EINVAL, "bad plk_params");
    if (cov_precision) *cov_precision = p.cov_precision;
    if (ps_da_max) *ps_da_max = p.ps_da_max;
    if (ref_scheme) *ref_scheme = p.ref_scheme;
    if (decay) *decay = p.decay;
    emi_params(p, ctx->work, out);
    if (alpha) *alpha = p.alpha;
    return PLK_OK;
}

extern "C" {

plk_status plk_default_params(plk_params *p) {
    if (!p) return fail(nullptr, PLK_EINVAL, "plk_default_params: null params");
    memset(p, 0, sizeof(*p));
    p->alpha = 1e-3;
    p->beta = 0.0f;
    p->mu = 0.99f;
    p->tol = 1e-6f;
    p->max_iter = 100;
    p->cond_max = 1e4f;
    p->fp64_resolve = 1;
    p->err_max = 0.1f;
    p->decay = 1.0f;
    return PLK_OK;
}

plk_status plk_output_shape(int H, int W, plk_window win, int *Ho, int *Wo) {
    if (!Ho || !Wo || H < 1 || W < 1 || !window_ok(win)) return fail(nullptr, PLK_EINVAL, "plk_output_shape: bad argument");
    *Ho = H / win.sy;
    *Wo = W / win.sx;
    return PLK_OK;
}

int plk_mask_words(plk_window win) { return (win.wy * win.wx + 63) / 64; }

plk_status plk_glrt_threshold(double alpha, int n_eff, double *c) {
    if (!c || !(alpha > 0.0 && alpha < 1.0) || n_eff < 1)
        return fail(nullptr, PLK_EINVAL, "plk_glrt_threshold: need 0 < alpha < 1, n_eff >= 1");
    return plk_glrt_threshold_looks(alpha, (double)n_eff, c);
}

plk_status plk_glrt_threshold_looks(double alpha, double nu, double *c) {
    if (!c || !(alpha > 0.0 && alpha < 1.0) || !(nu >= 1.0 && nu < 1e9))
        return fail(nullptr, PLK_EINVAL, "plk_glrt_threshold_looks: need 0 < alpha < 1, nu >= 1");
    // X = P_p / (P_p + P_q) ~ Beta(nu, nu); find x with I_x(nu, nu) = alpha / 2.
    const double a = nu, target = 0.5 * alpha;
    double lo = 0.0, hi = 0.5;
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (inc_beta_cf(a, a, mid) < target) lo = mid;
        else hi = mid;
    }
    const double x = 0.5 * (lo + hi);
    *c = (1.0 - x) / x;
    return PLK_OK;
}

plk_status plk_create(plk_ctx **out, int device, void *cuda_stream) {
    if (!out) return fail(nullptr, PLK_EINVAL, "plk_create: null out");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, PLK_ECUDA, "plk_create: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, PLK_EINVAL, "plk_create: device %d of %d", device, ndev);
    plk_ctx *ctx = new (std::nothrow) plk_ctx;
    if (!ctx) return fail(nullptr, PLK_ENOMEM, "plk_create: out of host memory");
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->err[0] = 0;
    ctx->n_agg = 0;
    ctx->n_tuned = 0;
    ctx->work = nullptr;
    {
        DeviceGuard dg(device);
        if (plk::dev_malloc((void **)&ctx->work, plk::kEmiWorkBytes) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return fail(nullptr, PLK_ENOMEM, "plk_create: device allocation failed");
        }
    }
    *out = ctx;
    return PLK_OK;
}

plk_status plk_destroy(plk_ctx *ctx) {
    if (!ctx) return PLK_OK;
    {
        DeviceGuard dg(ctx->device);
        if (ctx->prof.ev[0])
            for (int i = 0; i < 2 * plk::Prof::kMaxRecords; ++i) cudaEventDestroy(ctx->prof.ev[i]);
        cudaFree(ctx->work);
    }
    delete ctx;
    return PLK_OK;
}

plk_status plk_sync(plk_ctx *ctx) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_sync: null ctx");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_sync");
    if (plk::read_and_clear_wait_timeout())
        return fail(ctx, PLK_ETIMEOUT, "plk_sync: a device-side wait for staged tile data gave up");
    return PLK_OK;
}

plk_status plk_selftest_bounded_wait(plk_ctx *ctx) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_selftest_bounded_wait: null ctx");
    DeviceGuard dg(ctx->device);
    cudaError_t e = plk::launch_wait_selftest(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_selftest_bounded_wait");
    return PLK_OK;
}

plk_status plk_profile_enable(plk_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_profile_enable: null ctx");
    DeviceGuard dg(ctx->device);
    if (enable && !ctx->prof.ev[0]) {
        for (int i = 0; i < 2 * plk::Prof::kMaxRecords; ++i)
            if (cudaEventCreate(&ctx->prof.ev[i]) != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, PLK_ENOMEM, "plk_profile_enable: cudaEventCreate failed");
            }
    }
    ctx->prof.on = enable != 0;
    ctx->prof.n = 0;
    ctx->prof.overflow = false;
    return PLK_OK;
}

plk_status plk_profile_collect(plk_ctx *ctx, int *n_kernels) {
    if (!ctx || !n_kernels) return fail(ctx, PLK_EINVAL, "plk_profile_collect: bad argument");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_profile_collect");
    ctx->n_agg = 0;
    for (int i = 0; i < ctx->prof.n; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->prof.ev[2 * i], ctx->prof.ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int j = 0;
        while (j < ctx->n_agg && strcmp(ctx->agg_name[j], ctx->prof.name[i]) != 0) ++j;
        if (j == ctx->n_agg) {
            if (ctx->n_agg == 32) continue;
            ctx->agg_name[j] = ctx->prof.name[i];
            ctx->agg_ms[j] = 0.0;
            ctx->agg_count[j] = 0;
            ++ctx->n_agg;
        }
        ctx->agg_ms[j] += ms;
        ctx->agg_count[j] += 1;
    }
    const bool over = ctx->prof.overflow;
    ctx->prof.n = 0;
    ctx->prof.overflow = false;
    *n_kernels = ctx->n_agg;
    if (over) return fail(ctx, PLK_EINVAL, "plk_profile_collect: more than %d launches recorded", plk::Prof::kMaxRecords);
    return PLK_OK;
}

plk_status plk_profile_get(const plk_ctx *ctx, int i, const char **name, double *total_ms, int *launches) {
    if (!ctx || i < 0 || i >= ctx->n_agg || !name || !total_ms || !launches)
        return fail(nullptr, PLK_EINVAL, "plk_profile_get: bad argument");
    *name = ctx->agg_name[i];
    *total_ms = ctx->agg_ms[i];
    *launches = ctx->agg_count[i];
    return PLK_OK;
}

plk_status plk_set_stream(plk_ctx *ctx, void *cuda_stream) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_set_stream: null ctx");
    ctx->stream = (cudaStream_t)cuda_stream;
    return PLK_OK;
}

const char *plk_last_error(const plk_ctx *ctx) { return ctx ? ctx->err : g_noctx_err; }

plk_status plk_amp_stats(plk_ctx *ctx, const plk_c64 *slc, int n, int H, int W, float *sum_pow, float *sum_amp,
                         int accumulate) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_amp_stats: null ctx");
    if (!slc || !sum_pow || n < 1 || H < 1 || W < 1)
        return fail(ctx, PLK_EINVAL, "plk_amp_stats: bad argument");
    if (!aligned(slc, 8) || !aligned(sum_pow, 4) || (sum_amp && !aligned(sum_amp, 4)))
        return fail(ctx, PLK_EINVAL, "plk_amp_stats: misaligned pointer");
    DeviceGuard dg(ctx->device);
    ctx->prof.begin("amp_stats", ctx->stream);
    cudaError_t e = plk::launch_amp_stats(reinterpret_cast<const float2 *>(slc), n, (long long)H * W, sum_pow,
                                          sum_amp, accumulate, ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_amp_stats");
    return PLK_OK;
}

plk_status plk_shp_select(plk_ctx *ctx, const float *sum_pow, int n_eff, int H, int W, plk_window win,
                          double alpha, uint64_t *mask, uint16_t *count) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_shp_select: null ctx");
    if (!sum_pow || H < 1 || W < 1 || !window_ok(win) || n_eff < 1 || !(alpha > 0 && alpha < 1))
        return fail(ctx, PLK_EINVAL, "plk_shp_select: bad argument");
    if ((long long)(H / win.sy) * (W / win.sx) > 0 && (!mask || !count))
        return fail(ctx, PLK_EINVAL, "plk_shp_select: null output");
    if (!aligned(sum_pow, 4) || !aligned(mask, 8) || !aligned(count, 2))
        return fail(ctx, PLK_EINVAL, "plk_shp_select: misaligned pointer");
    double c;
    plk_glrt_threshold(alpha, n_eff, &c);
    DeviceGuard dg(ctx->device);
    const Geom g = plk::make_geom(H, W, win);
    ctx->prof.begin("shp_select", ctx->stream);
    cudaError_t e = plk::launch_shp(sum_pow, g, (float)c, mask, count, ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_shp_select");
    return PLK_OK;
}

plk_status plk_estimate_covariance(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                   const uint64_t *mask, int precision, plk_c64 *C_packed) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_estimate_covariance: null ctx");
    if (!slc || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || !window_ok(win) ||
        (precision != PLK_COV_FP32 && precision != PLK_COV_BF16 && precision != PLK_COV_FP16))
        return fail(ctx, PLK_EINVAL, "plk_estimate_covariance: bad argument");
    if (precision != PLK_COV_FP32 && N > 32)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_estimate_covariance: tensor-core modes need N <= 32 (N=%d)", N);
    if ((long long)(H / win.sy) * (W / win.sx) > 0 && (!mask || !C_packed))
        return fail(ctx, PLK_EINVAL, "plk_estimate_covariance: null pointer");
    if (!aligned(slc, 8) || !aligned(mask, 8) || !aligned(C_packed, 8))
        return fail(ctx, PLK_EINVAL, "plk_estimate_covariance: misaligned pointer");
    DeviceGuard dg(ctx->device);
    const Geom g = plk::make_geom(H, W, win);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    ctx->prof.begin("covariance", ctx->stream);
    cudaError_t e =
        plk::launch_covariance(z, N, g, mask, reinterpret_cast<float2 *>(C_packed), ctx->stream, precision);
    ctx->prof.end(ctx->stream);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_estimate_covariance: window %dx%d with N=%d exceeds shared memory",
                    win.wy, win.wx, N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_estimate_covariance");
    return PLK_OK;
}


plk_status plk_phase_link(plk_ctx *ctx, const plk_c64 *C_packed, int N, int64_t npx, int ref_idx,
                          const plk_params *params, float *phase, float *tcoh, float *lambda_min,
                          uint8_t *status) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_phase_link: null ctx");
    if (N < 2 || N > PLK_MAX_N || npx < 0 || ref_idx < 0 || ref_idx >= N)
        return fail(ctx, PLK_EINVAL, "plk_phase_link: bad argument");
    if (npx > 0 && (!C_packed || !phase || !status)) return fail(ctx, PLK_EINVAL, "plk_phase_link: null pointer");
    if (!aligned(C_packed, 8) || !aligned(phase, 4) || (tcoh && !aligned(tcoh, 4)) ||
        (lambda_min && !aligned(lambda_min, 4)))
        return fail(ctx, PLK_EINVAL, "plk_phase_link: misaligned pointer");
    plk::EmiParams prm;
    plk_status st = resolve_params(ctx, params, &prm, nullptr);
    if (st != PLK_OK) return st;
    DeviceGuard dg(ctx->device);
    cudaError_t e = plk::launch_phase_link(reinterpret_cast<const float2 *>(C_packed), N, npx, ref_idx, prm, phase,
                                           tcoh, lambda_min, status, ctx->stream, &ctx->prof);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_phase_link");
    return PLK_OK;
}

plk_status plk_compress(plk_ctx *ctx, const plk_c64 *slc, int N, int first_real, int H, int W, plk_window win,
                        const float *phase, plk_c64 *kappa) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_compress: null ctx");
    if (!slc || !phase || !kappa || N < 1 || N > PLK_MAX_N || first_real < 0 || first_real >= N || H < 1 ||
        W < 1 || !window_ok(win))
        return fail(ctx, PLK_EINVAL, "plk_compress: bad argument");
    if (!aligned(slc, 8) || !aligned(phase, 4) || !aligned(kappa, 8))
        return fail(ctx, PLK_EINVAL, "plk_compress: misaligned pointer");
    DeviceGuard dg(ctx->device);
    const Geom g = plk::make_geom(H, W, win);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    ctx->prof.begin("compress", ctx->stream);
    cudaError_t e =
        plk::launch_compress(z, N, first_real, g, phase, reinterpret_cast<float2 *>(kappa), ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_compress");
    return PLK_OK;
}

plk_status plk_ps_regrid(plk_ctx *ctx, const plk_c64 *slc, int N, int first_real, int H, int W, plk_window win,
                         const float *sum_pow, const float *sum_amp, int n_eff, int ref_idx, float da_max,
                         float *phase, uint8_t *status) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_ps_regrid: null ctx");
    if (N < 1 || N > PLK_MAX_N || first_real < 0 || first_real >= N || ref_idx < 0 || ref_idx >= N || H < 1 ||
        W < 1 || !window_ok(win) || n_eff < 1 || !(da_max >= 0.f && da_max < 1e30f))
        return fail(ctx, PLK_EINVAL, "plk_ps_regrid: bad argument");
    const Geom g = plk::make_geom(H, W, win);
    if ((long long)g.Ho * g.Wo == 0) return PLK_OK;
    if (!slc || !sum_pow || !sum_amp || !phase || !status) return fail(ctx, PLK_EINVAL, "plk_ps_regrid: null pointer");
    if (!aligned(slc, 8) || !aligned(sum_pow, 4) || !aligned(sum_amp, 4) || !aligned(phase, 4))
        return fail(ctx, PLK_EINVAL, "plk_ps_regrid: misaligned pointer");
    DeviceGuard dg(ctx->device);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    ctx->prof.begin("ps_regrid", ctx->stream);
    cudaError_t e = plk::launch_ps_regrid(z, N, first_real, ref_idx, g, sum_pow, sum_amp, n_eff, da_max, phase,
                                          status, ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ps_regrid");
    return PLK_OK;
}

plk_status plk_phase_similarity(plk_ctx *ctx, const float *phase, int M, int Ho, int Wo, int radius,
                                float *gamma_s) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_phase_similarity: null ctx");
    if (M < 2 || M > 32 || Ho < 0 || Wo < 0 || radius < 1 || radius > 32 || (long long)Ho * Wo >= (1LL << 31))
        return fail(ctx, PLK_EINVAL, "plk_phase_similarity: bad argument");
    if ((long long)Ho * Wo == 0) return PLK_OK;
    if (!phase || !gamma_s) return fail(ctx, PLK_EINVAL, "plk_phase_similarity: null pointer");
    if (!aligned(phase, 4) || !aligned(gamma_s, 4)) return fail(ctx, PLK_EINVAL, "plk_phase_similarity: misaligned pointer");
    DeviceGuard dg(ctx->device);
    ctx->prof.begin("phase_similarity", ctx->stream);
    cudaError_t e = plk::launch_phase_similarity(phase, M, Ho, Wo, radius, gamma_s, ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_phase_similarity: radius %d with M=%d exceeds shared memory", radius, M);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_phase_similarity");
    return PLK_OK;
}

plk_status plk_invert_l1(plk_ctx *ctx, const float *unw, int n_dates, const int32_t *pairs, int n_ifg, int64_t npx,
                         float rho, int iters, float *x, float *residual) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_invert_l1: null ctx");
    if (n_dates < 2 || n_ifg < 1 || npx < 0 || !pairs || !(rho > 0.f && rho < 1e30f) || iters < 1 ||
        iters > 100000)
        return fail(ctx, PLK_EINVAL, "plk_invert_l1: bad argument");
    if (n_dates > 17)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_invert_l1: %d dates (at most 17 are supported)", n_dates);
    const int nx = n_dates - 1;
    const int nxp = nx <= 4 ? 4 : nx <= 8 ? 8 : nx <= 12 ? 12 : nx;  // instantiated sizes: 4, 8, 12, 14, 15, 16
    if (nxp < 1) return fail(ctx, PLK_EINVAL, "plk_invert_l1: bad argument");
    plk::AdmmNet net;
    for (int s = 0; s < 48; ++s) net.plane[s] = -1;
    double G[16][16] = {};  // A^T A
    for (int k = 0; k < n_ifg; ++k) {
        const int a = pairs[2 * k], b = pairs[2 * k + 1];
        if (a < 0 || b >= n_dates || b <= a)
            return fail(ctx, PLK_EINVAL, "plk_invert_l1: pair %d = (%d, %d) is not 0 <= a < b < n_dates", k, a, b);
        if (b - a > 3)
            return fail(ctx, PLK_EUNSUPPORTED, "plk_invert_l1: pair %d = (%d, %d) is outside the nearest-3 network",
                        k, a, b);
        const int s = plk::admm_slot(nxp, b - a, a);
        if (net.plane[s] >= 0) return fail(ctx, PLK_EINVAL, "plk_invert_l1: pair (%d, %d) repeated", a, b);
        net.plane[s] = k;
        // row of A: -1 at date a, +1 at date b (date 0 dropped)
        const int ia = a - 1, ib = b - 1;
        G[ib][ib] += 1.0;
        if (ia >= 0) {
            G[ia][ia] += 1.0;
            G[ia][ib] -= 1.0;
            G[ib][ia] -= 1.0;
        }
    }
    // Banded Cholesky of A^T A (bandwidth 3 for these networks), identity beyond nx.
    double L[16][16] = {};
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j <= i; ++j) {
            double sum = G[i][j];
            for (int q = 0; q < j; ++q) sum -= L[i][q] * L[j][q];
            if (i == j) {
                if (!(sum > 1e-9))
                    return fail(ctx, PLK_EINVAL, "plk_invert_l1: the network does not determine date %d", i + 1);
                L[i][i] = sqrt(sum);
            } else {
                L[i][j] = sum / L[j][j];
            }
        }
    }
    for (int i = 0; i < 16; ++i) {
        net.L[i][0] = i < nx ? (float)(1.0 / L[i][i]) : 1.f;
        for (int q = 1; q <= 3; ++q) net.L[i][q] = (i < nx && i - q >= 0) ? (float)L[i][i - q] : 0.f;
    }
    net.kappa = 1.0f / rho;
    net.iters = iters;
    net.nx = nx;
    net.nxp = nxp;
    if (npx == 0) return PLK_OK;
    if (!unw || !x) return fail(ctx, PLK_EINVAL, "plk_invert_l1: null pointer");
    if (!aligned(unw, 4) || !aligned(x, 4) || (residual && !aligned(residual, 4)))
        return fail(ctx, PLK_EINVAL, "plk_invert_l1: misaligned pointer");
    DeviceGuard dg(ctx->device);
    ctx->prof.begin("invert_l1", ctx->stream);
    cudaError_t e = plk::launch_admm_l1(unw, npx, net, x, residual, ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_invert_l1");
    return PLK_OK;
}

// ----------------------------------------------------------------- adjoint

plk_status plk_backward_workspace_size(int N, int H, int W, plk_window win, size_t *bytes) {
    if (!bytes || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || !window_ok(win))
        return fail(nullptr, PLK_EINVAL, "plk_backward_workspace_size: bad argument");
    *bytes = plk::adjoint_workspace_bytes(N, plk::make_geom(H, W, win));
    return PLK_OK;
}

plk_status plk_phase_link_backward(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                   const uint64_t *mask, int ref_idx, const plk_params *params,
                                   const float *dphase, void *workspace, size_t workspace_bytes,
                                   plk_c64 *dslc) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_phase_link_backward: null ctx");
    if (!slc || !dslc || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || !window_ok(win) || ref_idx < 0 ||
        ref_idx >= N)
        return fail(ctx, PLK_EINVAL, "plk_phase_link_backward: bad argument");
    const plk::Geom g = plk::make_geom(H, W, win);
    const long long npx = (long long)g.Ho * g.Wo;
    if (npx > 0 && (!mask || !dphase || !workspace))
        return fail(ctx, PLK_EINVAL, "plk_phase_link_backward: null pointer");
    const size_t need = plk::adjoint_workspace_bytes(N, g);
    if (workspace_bytes < need)
        return fail(ctx, PLK_EINVAL, "plk_phase_link_backward: workspace of %zu bytes, %zu needed", workspace_bytes,
                    need);
    if (!aligned(slc, 8) || !aligned(dslc, 8) || !aligned(mask, 8) || !aligned(dphase, 4) ||
        !aligned(workspace, 256))
        return fail(ctx, PLK_EINVAL, "plk_phase_link_backward: misaligned pointer");
    plk::EmiParams prm;
    double alpha;
    plk_status ps = resolve_params(ctx, params, &prm, &alpha);
    if (ps != PLK_OK) return ps;
    DeviceGuard dg(ctx->device);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    cudaError_t e = plk::launch_adjoint(z, N, g, mask, ref_idx, prm, dphase, workspace,
                                        reinterpret_cast<float2 *>(dslc), ctx->stream, &ctx->prof);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_phase_link_backward: window with N=%d exceeds shared memory", N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_phase_link_backward");
    return PLK_OK;
}

plk_status plk_shp_weight_gradient(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                   const uint64_t *mask, int ref_idx, const plk_params *params,
                                   const float *dphase, void *workspace, size_t workspace_bytes, float *dweight) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_shp_weight_gradient: null ctx");
    if (!slc || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || !window_ok(win) || ref_idx < 0 || ref_idx >= N)
        return fail(ctx, PLK_EINVAL, "plk_shp_weight_gradient: bad argument");
    const plk::Geom g = plk::make_geom(H, W, win);
    const long long npx = (long long)g.Ho * g.Wo;
    if (npx > 0 && (!mask || !dphase || !workspace || !dweight))
        return fail(ctx, PLK_EINVAL, "plk_shp_weight_gradient: null pointer");
    const size_t need = plk::adjoint_workspace_bytes(N, g);
    if (workspace_bytes < need)
        return fail(ctx, PLK_EINVAL, "plk_shp_weight_gradient: workspace of %zu bytes, %zu needed", workspace_bytes,
                    need);
    if (!aligned(slc, 8) || !aligned(mask, 8) || !aligned(dphase, 4) || !aligned(dweight, 4) ||
        !aligned(workspace, 256))
        return fail(ctx, PLK_EINVAL, "plk_shp_weight_gradient: misaligned pointer");
    plk::EmiParams prm;
    double alpha;
    plk_status ps = resolve_params(ctx, params, &prm, &alpha);
    if (ps != PLK_OK) return ps;
    DeviceGuard dg(ctx->device);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    ctx->prof.begin("shp_weight_gradient", ctx->stream);
    cudaError_t e = plk::launch_weight_gradient(z, N, g, mask, ref_idx, prm, dphase, workspace, dweight,
                                                ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_shp_weight_gradient: window with N=%d exceeds shared memory", N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_shp_weight_gradient");
    return PLK_OK;
}

plk_status plk_phase_uncertainty(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                 const uint64_t *mask, int ref_idx, const plk_params *params, float sigma2,
                                 void *workspace, size_t workspace_bytes, float *phase_std) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_phase_uncertainty: null ctx");
    if (!slc || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || !window_ok(win) || ref_idx < 0 || ref_idx >= N ||
        !(sigma2 >= 0.f && sigma2 < 1e30f))
        return fail(ctx, PLK_EINVAL, "plk_phase_uncertainty: bad argument");
    const plk::Geom g = plk::make_geom(H, W, win);
    const long long npx = (long long)g.Ho * g.Wo;
    if (npx > 0 && (!mask || !workspace || !phase_std))
        return fail(ctx, PLK_EINVAL, "plk_phase_uncertainty: null pointer");
    const size_t need = plk::adjoint_workspace_bytes(N, g);
    if (workspace_bytes < need)
        return fail(ctx, PLK_EINVAL, "plk_phase_uncertainty: workspace of %zu bytes, %zu needed", workspace_bytes,
                    need);
    if (!aligned(slc, 8) || !aligned(mask, 8) || !aligned(phase_std, 4) || !aligned(workspace, 256))
        return fail(ctx, PLK_EINVAL, "plk_phase_uncertainty: misaligned pointer");
    plk::EmiParams prm;
    double alpha;
    plk_status ps = resolve_params(ctx, params, &prm, &alpha);
    if (ps != PLK_OK) return ps;
    DeviceGuard dg(ctx->device);
    Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * H * W;
    ctx->prof.begin("phase_uncertainty", ctx->stream);
    cudaError_t e = plk::launch_phase_uncertainty(z, N, g, mask, ref_idx, prm, sigma2, workspace, phase_std,
                                                  ctx->stream);
    ctx->prof.end(ctx->stream);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_phase_uncertainty: window with N=%d exceeds shared memory", N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_phase_uncertainty");
    return PLK_OK;
}

// ------------------------------------------------------------------- state

static void state_free(plk_state *st) {
    if (!st) return;
    if (st->ring) {
        for (int i = 0; i < st->K_max; ++i) cudaFree(st->ring[i]);
        free(st->ring);
    }
    cudaFree(st->sum_pow);
    cudaFree(st->sum_amp);
    cudaFree(st->da);
    cudaFree(st->amp_new);
    cudaFree(st->mask);
    cudaFree(st->count);
    cudaFree(st->C);
    cudaFree(st->phase_all);
    if (st->io.ready) {
        cudaStreamSynchronize(st->io.copy);
        for (int b = 0; b < 2; ++b) {
            cudaFree(st->io.stage[b]);
            cudaEventDestroy(st->io.copied[b]);
            cudaEventDestroy(st->io.released[b]);
        }
        cudaFree(st->io.phase);
        cudaFree(st->io.tcoh);
        cudaFree(st->io.status);
        cudaFree(st->io.count);
        cudaStreamDestroy(st->io.copy);
    }
    if (st->io.ready16)
        for (int b = 0; b < 2; ++b) {
            cudaFree(st->io.stage16[b]);
            cudaEventDestroy(st->io.widened[b]);
        }
    delete st;
}

plk_status plk_state_create(plk_ctx *ctx, int H, int W, plk_window win, int K_max, int M_max, plk_state **out) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_state_create: null ctx");
    if (!out || H < 1 || W < 1 || !window_ok(win) || K_max < 0 || M_max < 1 || K_max + M_max > PLK_MAX_N ||
        K_max + M_max < 2)
        return fail(ctx, PLK_EINVAL, "plk_state_create: bad argument");
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    plk_state *st = new (std::nothrow) plk_state;
    if (!st) return fail(ctx, PLK_ENOMEM, "plk_state_create: host");
    memset(st, 0, sizeof(*st));
    st->device = ctx->device;
    st->H = H;
    st->W = W;
    st->win = win;
    st->K_max = K_max;
    st->M_max = M_max;
    const Geom g = plk::make_geom(H, W, win);
    const long long npix = (long long)H * W, nout = (long long)g.Ho * g.Wo;
    const int Nmax = K_max + M_max;
    bool ok = true;
    st->ring = (float2 **)calloc(K_max > 0 ? K_max : 1, sizeof(float2 *));
    ok = ok && st->ring;
    for (int i = 0; ok && i < K_max; ++i) ok = plk::dev_malloc((void **)&st->ring[i], npix * sizeof(float2)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->sum_pow, npix * sizeof(float)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->sum_amp, npix * sizeof(float)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->da, npix * sizeof(float)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->amp_new, npix * sizeof(float)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->mask, (nout > 0 ? nout : 1) * g.nwords * sizeof(uint64_t)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->count, (nout > 0 ? nout : 1) * sizeof(uint16_t)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->C, (nout > 0 ? nout : 1) * plk::ntri(Nmax) * sizeof(float2)) == cudaSuccess;
    ok = ok && plk::dev_malloc((void **)&st->phase_all, (nout > 0 ? nout : 1) * Nmax * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMemsetAsync(st->sum_pow, 0, npix * sizeof(float), ctx->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(st->sum_amp, 0, npix * sizeof(float), ctx->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        state_free(st);
        return fail(ctx, PLK_ENOMEM, "plk_state_create: device allocation failed");
    }
    *out = st;
    return PLK_OK;
}

plk_status plk_state_destroy(plk_state *st) {
    if (!st) return PLK_OK;
    DeviceGuard dg(st->device);
    state_free(st);
    return PLK_OK;
}

plk_status plk_state_reset(plk_state *st) {
    if (!st) return fail(nullptr, PLK_EINVAL, "plk_state_reset: null state");
    st->K_used = 0;
    st->n_eff = 0;
    st->steps = 0;
    st->head = 0;
    st->W1 = st->W2 = 0.0;
    return PLK_OK;
}

plk_status plk_state_info(const plk_state *st, int *K_used, int *n_eff, int *steps) {
    if (!st) return fail(nullptr, PLK_EINVAL, "plk_state_info: null state");
    if (K_used) *K_used = st->K_used;
    if (n_eff) *n_eff = st->n_eff;
    if (steps) *steps = st->steps;
    return PLK_OK;
}

plk_status plk_state_weights(const plk_state *st, double *W1, double *W2) {
    if (!st) return fail(nullptr, PLK_EINVAL, "plk_state_weights: null state");
    if (W1) *W1 = st->W1;
    if (W2) *W2 = st->W2;
    return PLK_OK;
}

plk_status plk_state_kappa(const plk_state *st, int i, const plk_c64 **kappa) {
    if (!st || !kappa || i < 0 || i >= st->K_used) return fail(nullptr, PLK_EINVAL, "plk_state_kappa: bad argument");
    *kappa = reinterpret_cast<const plk_c64 *>(st->ring[(st->head + i) % st->K_max]);
    return PLK_OK;
}

plk_status plk_state_sums(const plk_state *st, const float **sum_pow, const float **sum_amp) {
    if (!st) return fail(nullptr, PLK_EINVAL, "plk_state_sums: null state");
    if (sum_pow) *sum_pow = st->sum_pow;
    if (sum_amp) *sum_amp = st->sum_amp;
    return PLK_OK;
}

// Format 2 adds the weight sums W1, W2 (two doubles) after the header;
// format 1 files (equal weights) load with W1 = W2 = n_eff.
static const char kMagic[8] = {'P', 'L', 'K', 'S', 'T', 'A', 'T', '2'};
static const char kMagic1[8] = {'P', 'L', 'K', 'S', 'T', 'A', 'T', '1'};

plk_status plk_state_save(plk_ctx *ctx, const plk_state *st, const char *path) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_state_save: null ctx");
    if (!st || !path) return fail(ctx, PLK_EINVAL, "plk_state_save: bad argument");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_state_save");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, PLK_EINVAL, "plk_state_save: cannot open %s", path);
    const long long npix = (long long)st->H * st->W;
    int32_t hdr[10] = {st->H, st->W, st->win.wy, st->win.wx, st->win.sy, st->win.sx,
                       st->K_max, st->K_used, st->n_eff, st->steps};
    const double wsum[2] = {st->W1, st->W2};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(wsum, sizeof(wsum), 1, f) == 1;
    void *host = malloc(npix * sizeof(float2));
    ok = ok && host;
    for (int i = 0; ok && i < st->K_used; ++i) {
        ok = cudaMemcpy(host, st->ring[(st->head + i) % st->K_max], npix * sizeof(float2), cudaMemcpyDeviceToHost) ==
                 cudaSuccess &&
             fwrite(host, sizeof(float2), npix, f) == (size_t)npix;
    }
    ok = ok && cudaMemcpy(host, st->sum_pow, npix * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
         fwrite(host, sizeof(float), npix, f) == (size_t)npix;
    ok = ok && cudaMemcpy(host, st->sum_amp, npix * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
         fwrite(host, sizeof(float), npix, f) == (size_t)npix;
    free(host);
    if (fclose(f) != 0) ok = false;
    if (!ok) return fail(ctx, PLK_ECUDA, "plk_state_save: write failed (%s)", path);
    return PLK_OK;
}

plk_status plk_state_load(plk_ctx *ctx, const char *path, int M_max, plk_state **out) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_state_load: null ctx");
    if (!path || !out) return fail(ctx, PLK_EINVAL, "plk_state_load: bad argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, PLK_EINVAL, "plk_state_load: cannot open %s", path);
    char magic[8];
    int32_t hdr[10];
    double wsum[2] = {0.0, 0.0};
    bool v2 = false;
    bool hdr_ok = fread(magic, 1, 8, f) == 8;
    if (hdr_ok) {
        v2 = memcmp(magic, kMagic, 8) == 0;
        hdr_ok = (v2 || memcmp(magic, kMagic1, 8) == 0) && fread(hdr, sizeof(hdr), 1, f) == 1;
    }
    if (hdr_ok && v2) hdr_ok = fread(wsum, sizeof(wsum), 1, f) == 1;
    if (!hdr_ok) {
        fclose(f);
        return fail(ctx, PLK_EINVAL, "plk_state_load: not a state file: %s", path);
    }
    if (!v2) wsum[0] = wsum[1] = hdr[8];
    plk_window win{hdr[2], hdr[3], hdr[4], hdr[5]};
    plk_state *st = nullptr;
    plk_status s = plk_state_create(ctx, hdr[0], hdr[1], win, hdr[6], M_max, &st);
    if (s != PLK_OK) {
        fclose(f);
        return s;
    }
    if (hdr[7] < 0 || hdr[7] > st->K_max) {
        fclose(f);
        plk_state_destroy(st);
        return fail(ctx, PLK_EINVAL, "plk_state_load: corrupt header");
    }
    DeviceGuard dg(ctx->device);
    const long long npix = (long long)st->H * st->W;
    void *host = malloc(npix * sizeof(float2));
    bool ok = host != nullptr && cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    for (int i = 0; ok && i < hdr[7]; ++i)
        ok = fread(host, sizeof(float2), npix, f) == (size_t)npix &&
             cudaMemcpy(st->ring[i], host, npix * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && fread(host, sizeof(float), npix, f) == (size_t)npix &&
         cudaMemcpy(st->sum_pow, host, npix * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && fread(host, sizeof(float), npix, f) == (size_t)npix &&
         cudaMemcpy(st->sum_amp, host, npix * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    free(host);
    fclose(f);
    if (!ok) {
        plk_state_destroy(st);
        return fail(ctx, PLK_EINVAL, "plk_state_load: truncated file %s", path);
    }
    st->K_used = hdr[7];
    st->n_eff = hdr[8];
    st->steps = hdr[9];
    st->W1 = wsum[0];
    st->W2 = wsum[1];
    st->head = 0;
    *out = st;
    return PLK_OK;
}

plk_status plk_ministack_step(plk_ctx *ctx, plk_state *st, const plk_c64 *new_slc, int M, const plk_params *params,
                              float *phase, float *tcoh, uint8_t *status, uint16_t *shp_count) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_ministack_step: null ctx");
    if (!st || !new_slc || M < 1 || M > st->M_max || st->K_used + M < 2)
        return fail(ctx, PLK_EINVAL, "plk_ministack_step: bad argument");
    const bool has_out = (long long)(st->H / st->win.sy) * (st->W / st->win.sx) > 0;
    if (has_out && (!phase || !tcoh || !status))
        return fail(ctx, PLK_EINVAL, "plk_ministack_step: null output");
    if (!aligned(new_slc, 8) || !aligned(phase, 4) || !aligned(tcoh, 4) || (shp_count && !aligned(shp_count, 2)))
        return fail(ctx, PLK_EINVAL, "plk_ministack_step: misaligned pointer");
    if (st->device != ctx->device) return fail(ctx, PLK_EINVAL, "plk_ministack_step: state on another device");
    plk::EmiParams prm;
    double alpha;
    int cov_precision = PLK_COV_FP32, ref_scheme = PLK_REF_FIRST;
    float ps_da_max = 0.f, decay = 1.f;
    plk_status ps = resolve_params(ctx, params, &prm, &alpha, &cov_precision, &ref_scheme, &ps_da_max, &decay);
    if (ps != PLK_OK) return ps;
    if (decay != 1.f && ps_da_max > 0.f)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_ministack_step: decaying weights with PS selection");
    if (cov_precision != PLK_COV_FP32 && st->K_used + M > 32)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_ministack_step: tensor-core coherence modes need N <= 32");
    DeviceGuard dg(ctx->device);
    const Geom g = plk::make_geom(st->H, st->W, st->win);
    const long long npix = (long long)st->H * st->W, nout = (long long)g.Ho * g.Wo;
    const int K = st->K_used, N = K + M;
    cudaStream_t s = ctx->stream;

    // S1: merge the new images into the running power sums.
    Planes znew{};
    for (int t = 0; t < M; ++t) znew.p[t] = reinterpret_cast<const float2 *>(new_slc) + (long long)t * npix;
    ctx->prof.begin("amp_stats", s);
    const int n_eff = st->n_eff + M;
    // With PS selection S1 also writes D_A of the merged sums (+inf where a new
    // sample is zero) and, at PS pixels, the amplitude sum of the new images.
    plk::PsStats pst;
    pst.da = st->da;
    pst.amp_new = st->amp_new;
    pst.n_eff = (float)n_eff;
    pst.da_max = ps_da_max;
    // Exponentially decaying weights (Sec. III-A): w_j = decay^(M-1-j) for the
    // new images, decay^M on the running sums, each a product of decays in
    // double precision rounded once to single precision; W1, W2 carried in
    // double precision.  decay = 1 takes the equal-weight path unchanged.
    double W1 = n_eff, W2 = n_eff;
    plk::SumWeights sw;
    if (decay != 1.f) {
        double acc = 1.0, w1 = 0.0, w2 = 0.0;
        for (int j = M - 1; j >= 0; --j) {
            sw.w[j] = (float)acc;
            w1 += (double)sw.w[j];
            w2 += (double)sw.w[j] * (double)sw.w[j];
            acc *= (double)decay;
        }
        sw.s = (float)acc;
        W1 = st->n_eff > 0 ? (double)sw.s * st->W1 + w1 : w1;
        W2 = st->n_eff > 0 ? (double)sw.s * (double)sw.s * st->W2 + w2 : w2;
    }
    cudaError_t e = plk::launch_amp_stats(reinterpret_cast<const float2 *>(new_slc), M, npix, st->sum_pow,
                                          st->sum_amp, st->n_eff > 0 ? 1 : 0, s, ps_da_max > 0.f ? &pst : nullptr,
                                          decay != 1.f ? &sw : nullptr);
    ctx->prof.end(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: amp_stats");

    // S2: SHP masks on the merged statistics (nu = W1^2 / W2 looks; n_eff at
    // equal weights).
    double c;
    if (decay != 1.f) plk_glrt_threshold_looks(alpha, W1 * W1 / W2 < 1.0 ? 1.0 : W1 * W1 / W2, &c);
    else plk_glrt_threshold(alpha, n_eff, &c);
    uint16_t *cnt = shp_count ? shp_count : st->count;
    ctx->prof.begin("shp_select", s);
    e = plk::launch_shp(st->sum_pow, g, (float)c, st->mask, cnt, s);
    ctx->prof.end(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: shp");

    // Mini-stack: compressed SLCs oldest..newest, then the new real SLCs.
    Planes z{};
    for (int i = 0; i < K; ++i) z.p[i] = st->ring[(st->head + i) % st->K_max];
    for (int t = 0; t < M; ++t) z.p[K + t] = znew.p[t];

    // S3-S6.
    ctx->prof.begin("covariance", s);
    e = plk::launch_covariance(z, N, g, st->mask, st->C, s, cov_precision);
    ctx->prof.end(s);
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, PLK_EUNSUPPORTED, "plk_ministack_step: window with N=%d exceeds shared memory", N);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: covariance");
    const int ref = K > 0 ? K - 1 : 0;
    const plk::StackSource src{&z, &g, st->mask};
    e = plk::launch_phase_link(st->C, N, nout, ref, prm, st->phase_all, tcoh, nullptr, status, s, &ctx->prof, &src);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: phase_link");
    if (nout > 0) {
        e = cudaMemcpyAsync(phase, st->phase_all + (long long)K * nout, (size_t)M * nout * sizeof(float),
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: phase copy");
    }
    // PS cells of the output take their PS's phases; below, each PS pixel is
    // compressed on its own phases, every other pixel on its cell's linked phases.
    if (ps_da_max > 0.f && nout > 0) {
        ctx->prof.begin("ps_regrid", s);
        e = plk::launch_ps_regrid(z, N, K, ref, g, nullptr, nullptr, n_eff, ps_da_max, phase, status, s, st->da);
        ctx->prof.end(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: ps_regrid");
    }

    // S7-S8: compress the real SLCs and push kappa into the ring.
    if (st->K_max > 0) {
        int slot;
        if (K < st->K_max) slot = (st->head + K) % st->K_max;
        else slot = st->head;
        ctx->prof.begin("compress", s);
        // PLK_REF_LAST_REAL: the new compressed SLC carries the last real date's phase.
        plk::PsSelect psel;
        if (ps_da_max > 0.f && nout > 0) {
            psel.da = st->da;
            psel.amp_new = st->amp_new;
            psel.da_max = ps_da_max;
            psel.ref = ref;
        }
        e = plk::launch_compress(z, N, K, g, st->phase_all, st->ring[slot], s,
                                 ref_scheme == PLK_REF_LAST_REAL ? N - 1 : -1, psel);
        ctx->prof.end(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step: compress");
        if (K < st->K_max) st->K_used = K + 1;
        else st->head = (st->head + 1) % st->K_max;
    }
    st->n_eff = n_eff;
    st->W1 = W1;
    st->W2 = W2;
    st->steps += 1;
    return PLK_OK;
}

plk_status plk_state_enable_host_io(plk_ctx *ctx, plk_state *st) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_state_enable_host_io: null ctx");
    if (!st) return fail(ctx, PLK_EINVAL, "plk_state_enable_host_io: null state");
    if (st->device != ctx->device) return fail(ctx, PLK_EINVAL, "plk_state_enable_host_io: state on another device");
    auto &io = st->io;
    if (io.ready) return PLK_OK;
    DeviceGuard dg(ctx->device);
    const long long npix = (long long)st->H * st->W;
    const long long nout = (long long)(st->H / st->win.sy) * (st->W / st->win.sx);
    memset(&io, 0, sizeof(io));
    const size_t nb = (size_t)st->M_max * npix * sizeof(float2), no = (size_t)(nout > 0 ? nout : 1);
    bool ok = plk::dev_malloc((void **)&io.stage[0], nb) == cudaSuccess &&
              plk::dev_malloc((void **)&io.stage[1], nb) == cudaSuccess &&
              plk::dev_malloc((void **)&io.phase, no * st->M_max * sizeof(float)) == cudaSuccess &&
              plk::dev_malloc((void **)&io.tcoh, no * sizeof(float)) == cudaSuccess &&
              plk::dev_malloc((void **)&io.status, no) == cudaSuccess &&
              plk::dev_malloc((void **)&io.count, no * sizeof(uint16_t)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&io.copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < 2; ++b)
        ok = cudaEventCreateWithFlags(&io.copied[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&io.released[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(io.stage[b]);
            if (io.copied[b]) cudaEventDestroy(io.copied[b]);
            if (io.released[b]) cudaEventDestroy(io.released[b]);
        }
        cudaFree(io.phase);
        cudaFree(io.tcoh);
        cudaFree(io.status);
        cudaFree(io.count);
        if (io.copy) cudaStreamDestroy(io.copy);
        memset(&io, 0, sizeof(io));
        cudaGetLastError();
        return fail(ctx, PLK_ENOMEM, "plk_state_enable_host_io: cannot allocate %zu bytes of staging", 2 * nb);
    }
    io.ready = true;
    return PLK_OK;
}

int64_t plk_device_allocations(void) { return plk::g_device_allocations.load(std::memory_order_relaxed); }

namespace {

// Steps of plk_ministack_step_host[_ci16] after the call's SLCs are in
// stage[b] (stream-ordered on ctx's stream): the step itself, the release of
// stage[b], and the outputs' copies to host memory.
plk_status step_from_stage(plk_ctx *ctx, plk_state *st, int b, int M, const plk_params *params, float *phase,
                           float *tcoh, uint8_t *status, uint16_t *shp_count, const char *who) {
    auto &io = st->io;
    const long long nout = (long long)(st->H / st->win.sy) * (st->W / st->win.sx);
    plk_status ps = plk_ministack_step(ctx, st, reinterpret_cast<const plk_c64 *>(io.stage[b]), M, params, io.phase,
                                       io.tcoh, io.status, shp_count ? io.count : nullptr);
    if (ps != PLK_OK) return ps;
    cudaError_t e = cudaEventRecord(io.released[b], ctx->stream);
    if (e == cudaSuccess && nout > 0) {
        e = cudaMemcpyAsync(phase, io.phase, (size_t)M * nout * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tcoh, io.tcoh, (size_t)nout * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(status, io.status, (size_t)nout, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && shp_count)
            e = cudaMemcpyAsync(shp_count, io.count, (size_t)nout * sizeof(uint16_t), cudaMemcpyDeviceToHost,
                                ctx->stream);
    }
    if (e != cudaSuccess) {
        char what[96];
        snprintf(what, sizeof what, "%s: output copy", who);
        return cuda_fail(ctx, e, what);
    }
    return PLK_OK;
}

// Argument checks shared by the two host-buffer steps.
plk_status check_host_step(plk_ctx *ctx, plk_state *st, const void *new_slc, int M, float *phase, float *tcoh,
                           uint8_t *status, bool need16, const char *who) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "%s: null ctx", who);
    if (!st || !new_slc || M < 1 || M > st->M_max || st->K_used + M < 2)
        return fail(ctx, PLK_EINVAL, "%s: bad argument", who);
    if (st->device != ctx->device) return fail(ctx, PLK_EINVAL, "%s: state on another device", who);
    const long long nout = (long long)(st->H / st->win.sy) * (st->W / st->win.sx);
    if (nout > 0 && (!phase || !tcoh || !status)) return fail(ctx, PLK_EINVAL, "%s: null output", who);
    if (!st->io.ready || (need16 && !st->io.ready16))
        return fail(ctx, PLK_EINVAL, "%s: no staging; call plk_state_enable_host_io%s first", who, need16 ? "_ci16" : "");
    return PLK_OK;
}

}  // namespace

plk_status plk_ministack_step_host(plk_ctx *ctx, plk_state *st, const plk_c64 *new_slc, int M,
                                   const plk_params *params, float *phase, float *tcoh, uint8_t *status,
                                   uint16_t *shp_count) {
    const char *who = "plk_ministack_step_host";
    plk_status ps = check_host_step(ctx, st, new_slc, M, phase, tcoh, status, false, who);
    if (ps != PLK_OK) return ps;
    DeviceGuard dg(ctx->device);
    auto &io = st->io;
    const long long npix = (long long)st->H * st->W;
    const int b = io.next;
    io.next ^= 1;
    // Copy stream: wait until the step that last read stage[b] has run, then copy.
    cudaError_t e = cudaStreamWaitEvent(io.copy, io.released[b], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(io.stage[b], new_slc, (size_t)M * npix * sizeof(float2), cudaMemcpyHostToDevice, io.copy);
    if (e == cudaSuccess) e = cudaEventRecord(io.copied[b], io.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, io.copied[b], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step_host: staging copy");
    return step_from_stage(ctx, st, b, M, params, phase, tcoh, status, shp_count, who);
}

plk_status plk_state_enable_host_io_ci16(plk_ctx *ctx, plk_state *st) {
    plk_status ps = plk_state_enable_host_io(ctx, st);
    if (ps != PLK_OK) return ps;
    auto &io = st->io;
    if (io.ready16) return PLK_OK;
    DeviceGuard dg(ctx->device);
    const size_t nb = (size_t)st->M_max * st->H * st->W * 2 * sizeof(int16_t);
    io.stage16[0] = io.stage16[1] = nullptr;
    io.widened[0] = io.widened[1] = nullptr;
    bool ok = plk::dev_malloc((void **)&io.stage16[0], nb) == cudaSuccess &&
              plk::dev_malloc((void **)&io.stage16[1], nb) == cudaSuccess;
    for (int b = 0; ok && b < 2; ++b)
        ok = cudaEventCreateWithFlags(&io.widened[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(io.stage16[b]);
            if (io.widened[b]) cudaEventDestroy(io.widened[b]);
            io.stage16[b] = nullptr;
            io.widened[b] = nullptr;
        }
        cudaGetLastError();
        return fail(ctx, PLK_ENOMEM, "plk_state_enable_host_io_ci16: cannot allocate %zu bytes of staging", 2 * nb);
    }
    io.ready16 = true;
    return PLK_OK;
}

plk_status plk_ministack_step_host_ci16(plk_ctx *ctx, plk_state *st, const int16_t *new_slc, int M,
                                        const plk_params *params, float *phase, float *tcoh, uint8_t *status,
                                        uint16_t *shp_count) {
    const char *who = "plk_ministack_step_host_ci16";
    plk_status ps = check_host_step(ctx, st, new_slc, M, phase, tcoh, status, true, who);
    if (ps != PLK_OK) return ps;
    if ((uintptr_t)new_slc % 4) return fail(ctx, PLK_EINVAL, "%s: new_slc not 4-byte aligned", who);
    DeviceGuard dg(ctx->device);
    auto &io = st->io;
    const long long n = (long long)M * st->H * st->W;  // complex samples
    const int b = io.next;
    io.next ^= 1;
    // Copy stream: wait until stage16[b] has been widened for its last step, then copy.
    cudaError_t e = cudaStreamWaitEvent(io.copy, io.widened[b], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(io.stage16[b], new_slc, (size_t)n * 2 * sizeof(int16_t), cudaMemcpyHostToDevice, io.copy);
    if (e == cudaSuccess) e = cudaEventRecord(io.copied[b], io.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, io.copied[b], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step_host_ci16: staging copy");
    // Widen into stage[b] on ctx's stream (after the step that last read it, in stream order).
    e = plk::launch_ci16_to_c64(io.stage16[b], io.stage[b], n, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(io.widened[b], ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_ministack_step_host_ci16: widening");
    return step_from_stage(ctx, st, b, M, params, phase, tcoh, status, shp_count, who);
}

}  // extern "C"
