// S7. Compressed SLC (Sec. II-B): kappa = zeta^H z over the real SLCs, each
// full-resolution pixel using the linked phases of the output cell whose
// decimation block contains it (optionally re-referenced to one date, whose
// phase is subtracted: the last-real-SLC scheme) (the last cell row/column also takes the rows
// and columns beyond the output grid).
//
// A block owns one output row's decimation rows (sy rows, or the remainder for
// the last output row) times 256 image columns.  It first turns the phases of
// the cells its columns fall in into unit phasors exp(-j phi) in shared memory
// (one sincosf per cell and date, not per pixel), then streams the pixels:
// one thread per column, eight dates in flight per thread.  HBM-streaming.
//
// With PS selection on, a persistent scatterer is compressed on its own
// phases theta_i = arg(z_i conj z_ref) (minus theta at shift_date when
// re-referenced) instead of its cell's: then every term conj(zeta_i) z_i is
// |z_i| times the unit phasor u of z_ref (of z at shift_date), so
// kappa = (sum_i |z_i|) u, and the next mini-stack's PS phases keep the datum.
// The amplitude sum over the real dates is the one S1 took for them.
#include <algorithm>

#include "ps.cuh"

namespace plk {

constexpr int kCompressCols = 256;

// Cells one block's columns can touch: 256 / sx + 2 at most.
static int max_cells(int sx) { return kCompressCols / sx + 2; }

template <bool PS>
__global__ void __launch_bounds__(kCompressCols) k_compress(const __grid_constant__ Planes z, int n, int first_real,
                                                           const Geom g, const float *__restrict__ phase,
                                                           float2 *__restrict__ kappa, int nchunk,
                                                           int shift_date, const PsSelect ps) {
    extern __shared__ float2 ph[];  // (n - first_real) x ncell phasors, date-major
    const long long nout = (long long)g.Ho * g.Wo;
    const int nr = n - first_real;
    const long long nblocks = (long long)g.Ho * nchunk;
    for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int ci = (int)(b / nchunk), chunk = (int)(b - (long long)ci * nchunk);
        const int X0 = chunk * kCompressCols;
        const int y_lo = ci * g.sy, y_hi = (ci == g.Ho - 1) ? g.H : y_lo + g.sy;
        const int c_lo = min(X0 / g.sx, g.Wo - 1);
        const int c_hi = min(min(X0 + kCompressCols - 1, g.W - 1) / g.sx, g.Wo - 1);
        const int ncell = c_hi - c_lo + 1;
        __syncthreads();  // the previous block's phasors are no longer read
        for (int idx = threadIdx.x; idx < nr * ncell; idx += blockDim.x) {
            const int i = idx / ncell, c = idx - i * ncell;
            const long long cell = (long long)ci * g.Wo + c_lo + c;
            float v = __ldg(phase + (long long)(first_real + i) * nout + cell);
            // re-referenced to date shift_date when asked (its phase subtracted)
            if (shift_date >= 0) v -= __ldg(phase + (long long)shift_date * nout + cell);
            float s, cs;
            sincosf(v, &s, &cs);  // NaN phase -> NaN phasor -> pixel marked bad
            ph[idx] = make_float2(cs, s);
        }
        __syncthreads();
        const int x = X0 + threadIdx.x;
        if (x >= g.W) continue;
        const int c = min(x / g.sx, g.Wo - 1) - c_lo;
        for (int y = y_lo; y < y_hi; ++y) {
            const long long q = (long long)y * g.W + x;
            float kr = 0.f, ki = 0.f;
            float2 last = make_float2(0.f, 0.f);  // PS: the last real date's sample
            bool bad = false;
            int i = 0;
            for (; i + 8 <= nr; i += 8) {
                float2 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcs(z.p[first_real + i + u] + q);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 e = ph[(i + u) * ncell + c];
                    bad |= isnan(e.x);
                    // exp(-j phi) * v
                    kr += e.x * v[u].x + e.y * v[u].y;
                    ki += e.x * v[u].y - e.y * v[u].x;
                }
                if (PS) last = v[7];
            }
            for (; i < nr; ++i) {
                const float2 e = ph[i * ncell + c];
                const float2 v = __ldcs(z.p[first_real + i] + q);
                bad |= isnan(e.x);
                kr += e.x * v.x + e.y * v.y;
                ki += e.x * v.y - e.y * v.x;
                if (PS) last = v;
            }
            if (PS && __ldg(ps.da + q) <= ps.da_max && ref_sample_nonzero(z, ps.ref, q)) {
                // a PS: compressed on its own phases, kappa = (sum |z_i|) u
                const float2 u = shift_date == n - 1 ? last : __ldg(z.p[shift_date >= 0 ? shift_date : ps.ref] + q);
                const float sc = __ldg(ps.amp_new + q) * rhypotf(u.x, u.y);
                kappa[q] = make_float2(u.x * sc, u.y * sc);
                continue;
            }
            kappa[q] = bad ? make_float2(0.f, 0.f) : make_float2(kr, ki);
        }
    }
}

cudaError_t launch_compress(const Planes &z, int n, int first_real, const Geom &g, const float *phase,
                            float2 *kappa, cudaStream_t s, int shift_date, const PsSelect &ps) {
    const long long npix = (long long)g.H * g.W;
    if (npix == 0) return cudaSuccess;
    if (g.Ho == 0 || g.Wo == 0) return cudaMemsetAsync(kappa, 0, npix * sizeof(float2), s);
    const int nchunk = (g.W + kCompressCols - 1) / kCompressCols;
    const size_t smem = (size_t)std::max(n - first_real, 1) * max_cells(g.sx) * sizeof(float2);
    auto kern = ps.da != nullptr ? k_compress<true> : k_compress<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long nblocks = (long long)g.Ho * nchunk;
    const long long grid = std::min<long long>(nblocks, (long long)device_sm_count() * 64);
    kern<<<(unsigned)grid, kCompressCols, smem, s>>>(z, n, first_real, g, phase, kappa, nchunk, shift_date, ps);
    return cudaGetLastError();
}

}  // namespace plk
