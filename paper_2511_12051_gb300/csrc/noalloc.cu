// plk_phase_link_stack_noalloc: one mini-stack through S1-S6 without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Its working buffers (power sums, SHP masks and counts, packed coherence)
// live in one file-scope __device__ array of PLK_NOALLOC_SCRATCH_BYTES.  Host
// code cannot use the array's name as a device address: every call looks the
// address up with cudaGetSymbolAddress, with the calling device current, so
// the address always belongs to that device's present context (a cached one
// would be stale after the context is torn down and made again).
#include <stdio.h>
#include <string.h>

#include "api_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PLK_NOALLOC_SCRATCH_BYTES];

// Errors are reported through plk_last_error(NULL), like other calls without a context.
plk_status fail(plk_status st, const char *msg) {
    plk::set_noctx_error(msg);
    return st;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" plk_status plk_phase_link_stack_noalloc(const plk_c64 *slc, int N, int H, int W, plk_window win,
                                                   int ref_idx, const plk_params *params, float *phase,
                                                   float *tcoh, uint8_t *status, uint16_t *shp_count,
                                                   void *cuda_stream) {
    if (!slc || N < 2 || N > PLK_MAX_N || H < 1 || W < 1 || ref_idx < 0 || ref_idx >= N || win.wy < 1 ||
        win.wx < 1 || !(win.wy & 1) || !(win.wx & 1) || win.sy < 1 || win.sx < 1 ||
        (long long)win.wy * win.wx > PLK_MAX_WINDOW)
        return fail(PLK_EINVAL, "plk_phase_link_stack_noalloc: bad argument");
    const plk::Geom g = plk::make_geom(H, W, win);
    const long long npix = (long long)H * W, nout = (long long)g.Ho * g.Wo;
    if (nout > 0 && (!phase || !tcoh || !status))
        return fail(PLK_EINVAL, "plk_phase_link_stack_noalloc: null output");
    if (((uintptr_t)slc % 8) || (phase && ((uintptr_t)phase % 4)) || (tcoh && ((uintptr_t)tcoh % 4)) ||
        (shp_count && ((uintptr_t)shp_count % 2)))
        return fail(PLK_EINVAL, "plk_phase_link_stack_noalloc: misaligned pointer");

    // Scratch layout: re-solve work area | sums [H][W] float | mask [Ho][Wo][words] | counts | C.
    // Every region takes at least a byte per pixel, so sizes past the limit are
    // refused before any product is formed (no wrap-around in the sum below).
    const size_t cap = (size_t)PLK_NOALLOC_SCRATCH_BYTES;
    const size_t b_work = align256(plk::kEmiWorkBytes);
    size_t need = cap + 1;
    if ((size_t)npix <= cap && (size_t)nout <= cap) {
        const size_t b_pow = align256((size_t)npix * sizeof(float));
        const size_t b_mask = align256((size_t)nout * g.nwords * sizeof(uint64_t));
        const size_t b_cnt = align256((size_t)nout * sizeof(uint16_t));
        const size_t b_c = align256((size_t)nout * plk::ntri(N) * sizeof(float2));
        need = b_work + b_pow + b_mask + b_cnt + b_c;
    }
    if (need > cap) {
        char msg[256];
        if (need == cap + 1)
            snprintf(msg, sizeof msg,
                     "plk_phase_link_stack_noalloc: N=%d, %dx%d needs more scratch than the limit of %zu bytes "
                     "(PLK_NOALLOC_SCRATCH_BYTES)",
                     N, H, W, cap);
        else
            snprintf(msg, sizeof msg,
                     "plk_phase_link_stack_noalloc: needs %zu bytes of scratch for N=%d, %dx%d; the limit is %zu "
                     "(PLK_NOALLOC_SCRATCH_BYTES)",
                     need, N, H, W, cap);
        return fail(PLK_EINVAL, msg);
    }
    const size_t b_pow = align256((size_t)npix * sizeof(float));
    const size_t b_mask = align256((size_t)nout * g.nwords * sizeof(uint64_t));
    const size_t b_cnt = align256((size_t)nout * sizeof(uint16_t));
    plk_params p;
    if (params) p = *params;
    else plk_default_params(&p);
    if (!plkapi::params_ok(p)) return fail(PLK_EINVAL, "plk_phase_link_stack_noalloc: bad plk_params");
    if (p.ps_da_max > 0.f)
        return fail(PLK_EUNSUPPORTED,
                    "plk_phase_link_stack_noalloc: no persistent-scatterer regridding (ps_da_max must be 0)");
    if (p.cov_precision != PLK_COV_FP32 && N > 32)
        return fail(PLK_EUNSUPPORTED, "plk_phase_link_stack_noalloc: tensor-core coherence modes need N <= 32");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: no current CUDA device");
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
        cudaGetLastError();
        return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: cudaGetSymbolAddress failed");
    }
    unsigned char *base = static_cast<unsigned char *>(addr);
    unsigned long long *work = reinterpret_cast<unsigned long long *>(base);
    base += b_work;
    float *sum_pow = reinterpret_cast<float *>(base);
    uint64_t *mask = reinterpret_cast<uint64_t *>(base + b_pow);
    uint16_t *cnt = shp_count ? shp_count : reinterpret_cast<uint16_t *>(base + b_pow + b_mask);
    float2 *C = reinterpret_cast<float2 *>(base + b_pow + b_mask + b_cnt);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    plk::EmiParams prm;
    plkapi::emi_params(p, work, &prm);

    // Every scratch region is written in full before it is read in this call.
    e = plk::launch_amp_stats(reinterpret_cast<const float2 *>(slc), N, npix, sum_pow, nullptr, 0, s);
    if (e != cudaSuccess) return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: amp_stats launch failed");
    double c;
    plk_glrt_threshold(p.alpha, N, &c);
    e = plk::launch_shp(sum_pow, g, (float)c, mask, cnt, s);
    if (e != cudaSuccess) return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: shp launch failed");
    plk::Planes z{};
    for (int t = 0; t < N; ++t) z.p[t] = reinterpret_cast<const float2 *>(slc) + (long long)t * npix;
    e = plk::launch_covariance(z, N, g, mask, C, s, p.cov_precision);
    if (e == cudaErrorInvalidConfiguration)
        return fail(PLK_EUNSUPPORTED, "plk_phase_link_stack_noalloc: window too large for shared memory");
    if (e != cudaSuccess) return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: covariance launch failed");
    const plk::StackSource src{&z, &g, mask};
    e = plk::launch_phase_link(C, N, nout, ref_idx, prm, phase, tcoh, nullptr, status, s, nullptr, &src);
    if (e != cudaSuccess) return fail(PLK_ECUDA, "plk_phase_link_stack_noalloc: phase_link launch failed");
    return PLK_OK;
}
