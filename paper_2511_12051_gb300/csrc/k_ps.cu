// Persistent scatterers (Sec. III-A, amplitude dispersion D_A = sigma_A / mu_A;
// Sec. IV, threshold on D_A at full resolution) and their regridding onto the
// output grid (Supplement, "Regridding PS and DS to 30 m resolution"): a cell
// whose decimation block holds PS takes the single-reference phase of the one
// with the lowest D_A; a cell without PS keeps its phase-linking result.
//
// A PS also needs nonzero samples at the reference entry and on every real
// date, so that each of its phases arg(z_i conj z_ref) is defined.
//
// One thread per output cell.  Threads of a warp own consecutive cells of one
// output row, so each row of their blocks is one contiguous run of the input
// planes (coalesced).  D_A is taken in single precision with correctly rounded
// operations in one fixed order, so the PS decision is reproducible bit for
// bit by any IEEE single-precision implementation of the same formula.
//
// Two sources of D_A: the merged sums (FROM_SUMS; the real samples of each
// candidate are then read to check them), or the plane the S1 kernel wrote
// inside a mini-stack step, where a zero real sample already gives +inf and a
// candidate costs one read, its reference sample.  The chosen PS's samples are
// read with eight dates in flight.
#include "ps.cuh"

namespace plk {

template <bool FROM_SUMS>
__device__ __forceinline__ float cell_da(const float *__restrict__ src0, const float *__restrict__ src1, float n_eff,
                                         long long q) {
    return FROM_SUMS ? amp_dispersion(__ldg(src0 + q), __ldg(src1 + q), n_eff) : __ldg(src0 + q);
}

template <bool FROM_SUMS>
__device__ __forceinline__ bool cell_ok(const Planes &z, int n, int first_real, int ref, long long q) {
    return FROM_SUMS ? ps_samples_nonzero(z, n, first_real, ref, q) : ref_sample_nonzero(z, ref, q);
}

// One thread per output cell (no grid-stride: the grid covers every cell).
template <bool FROM_SUMS>
__global__ void __launch_bounds__(256) k_ps_regrid(const __grid_constant__ Planes z, int n, int first_real, int ref,
                                                   const Geom g, const float *__restrict__ src0,
                                                   const float *__restrict__ src1, float n_eff, float da_max,
                                                   float *__restrict__ phase, uint8_t *__restrict__ status) {
    const long long nout = (long long)g.Ho * g.Wo;
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= nout) return;
    const int ci = (int)(cell / g.Wo), cj = (int)(cell - (long long)ci * g.Wo);
    const int y_lo = ci * g.sy, y_hi = (ci == g.Ho - 1) ? g.H : y_lo + g.sy;
    const int x_lo = cj * g.sx, x_hi = (cj == g.Wo - 1) ? g.W : x_lo + g.sx;
    // The lowest D_A within the threshold (strictly lower: the first in
    // row-major order wins a tie), from the dispersions alone; then the
    // sample check of that pixel.  Only if it fails (a zero sample) is the
    // block scanned again with the check on every candidate: the same choice.
    float best = __int_as_float(0x7f800000);  // +inf
    long long bq = -1;
    for (int y = y_lo; y < y_hi; ++y) {
#pragma unroll 4
        for (int x = x_lo; x < x_hi; ++x) {
            const long long q = (long long)y * g.W + x;
            const float da = cell_da<FROM_SUMS>(src0, src1, n_eff, q);
            if (da <= da_max && da < best) {
                best = da;
                bq = q;
            }
        }
    }
    if (bq < 0) return;
    if (!cell_ok<FROM_SUMS>(z, n, first_real, ref, bq)) {
        best = __int_as_float(0x7f800000);
        bq = -1;
        for (int y = y_lo; y < y_hi; ++y) {
            for (int x = x_lo; x < x_hi; ++x) {
                const long long q = (long long)y * g.W + x;
                const float da = cell_da<FROM_SUMS>(src0, src1, n_eff, q);
                if (da <= da_max && da < best && cell_ok<FROM_SUMS>(z, n, first_real, ref, q)) {
                    best = da;
                    bq = q;
                }
            }
        }
        if (bq < 0) return;
    }
    const float2 r = __ldg(z.p[ref] + bq);
    const int nr = n - first_real;
    for (int j0 = 0; j0 < nr; j0 += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u < nr) v[u] = __ldg(z.p[first_real + j0 + u] + bq);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (j0 + u >= nr) break;
            // v conj(r), rounded as written (exact zero imaginary part at the reference)
            const float re = __fadd_rn(__fmul_rn(v[u].x, r.x), __fmul_rn(v[u].y, r.y));
            const float im = __fsub_rn(__fmul_rn(v[u].y, r.x), __fmul_rn(v[u].x, r.y));
            phase[(long long)(j0 + u) * nout + cell] = atan2f(im, re);
        }
    }
    status[cell] = PLK_PX_PS;
}

cudaError_t launch_ps_regrid(const Planes &z, int n, int first_real, int ref, const Geom &g, const float *sum_pow,
                             const float *sum_amp, int n_eff, float da_max, float *phase, uint8_t *status,
                             cudaStream_t s, const float *da) {
    const long long nout = (long long)g.Ho * g.Wo;
    if (nout <= 0) return cudaSuccess;
    const long long grid = (nout + 255) / 256;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (da)
        k_ps_regrid<false><<<(unsigned)grid, 256, 0, s>>>(z, n, first_real, ref, g, da, nullptr, 0.f, da_max, phase,
                                                          status);
    else
        k_ps_regrid<true><<<(unsigned)grid, 256, 0, s>>>(z, n, first_real, ref, g, sum_pow, sum_amp, (float)n_eff,
                                                         da_max, phase, status);
    return cudaGetLastError();
}

}  // namespace plk
