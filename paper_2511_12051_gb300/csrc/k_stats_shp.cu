// S1 amplitude statistics and S2 GLRT SHP selection (Sec. III-A).
//
// Both kernels are HBM-streaming: one thread per pixel, coalesced 8-byte loads
// across a warp, grid sized in multiples of the SM count.  The power sums and
// the threshold product decide mask bits, so they use explicitly rounded
// single-precision operations (__fmul_rn / __fadd_rn, never contracted into
// an FMA) in one fixed order.
//
// With PS outputs, S1 also writes D_A of the merged sums per pixel (Sec.
// III-A) where it is within the threshold or near it, +inf elsewhere and where
// one of the new samples is zero, and, at the pixels with D_A <= da_max, this
// mini-stack's amplitude sum: the PS test of the
// regridding and compression passes then reads one float per pixel and no
// samples, and compression reads the amplitude sum at PS pixels only.
#include <algorithm>

#include "ps.cuh"

namespace plk {

template <bool DA>
__global__ void __launch_bounds__(256, 8) k_amp_stats(const float2 *__restrict__ z, int n, long long npix,
                                                   float *__restrict__ sum_pow, float *__restrict__ sum_amp,
                                                   int accumulate, const PsStats ps) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
        float P = 0.0f, A = 0.0f;
        bool nz = true;  // every new sample nonzero
        int t = 0;
        // Eight dates in flight per thread; the sums still run in date order.
        for (; t + 8 <= n; t += 8) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(z + (long long)(t + u) * npix + p);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float q = __fadd_rn(__fmul_rn(v[u].x, v[u].x), __fmul_rn(v[u].y, v[u].y));
                P = __fadd_rn(P, q);
                A = __fadd_rn(A, __fsqrt_rn(q));
                if (DA) nz &= (v[u].x != 0.f) | (v[u].y != 0.f);
            }
        }
        for (; t < n; ++t) {
            const float2 v = __ldcs(z + (long long)t * npix + p);
            const float q = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
            P = __fadd_rn(P, q);
            A = __fadd_rn(A, __fsqrt_rn(q));
            if (DA) nz &= (v.x != 0.f) | (v.y != 0.f);
        }
        const float A_new = A;
        if (accumulate) {
            P = __fadd_rn(sum_pow[p], P);
            if (sum_amp) A = __fadd_rn(sum_amp[p], A);
        }
        sum_pow[p] = P;
        if (sum_amp) sum_amp[p] = A;
        if (DA) {
            // D_A exactly (amp_dispersion's operations) where it can be within
            // the threshold; +inf where n SP - SA^2 exceeds (1.001 da_max SA)^2,
            // a margin far above the rounding of either side, so that every
            // pixel with exact D_A <= da_max keeps its value.
            float d = __int_as_float(0x7f800000);
            if (nz && A > 0.f) {
                const float num2 = fmaxf(__fsub_rn(__fmul_rn(ps.n_eff, P), __fmul_rn(A, A)), 0.f);
                const float lim = 1.001f * ps.da_max * A;
                if (num2 <= lim * lim) d = amp_dispersion(P, A, ps.n_eff);
            }
            ps.da[p] = d;
            if (d <= ps.da_max) ps.amp_new[p] = A_new;
        }
    }
}

// S1 with exponentially decaying image weights (Sec. III-A): per pixel
// P_g = sum_j fl(w_j q_j), A_g = sum_j fl(w_j sqrt(q_j)), j ascending, and the
// running sums become fl(fl(s P) + P_g), fl(fl(s A) + A_g).  Same rounding
// discipline as k_amp_stats (the sums decide mask bits).
__global__ void __launch_bounds__(256, 8) k_amp_stats_w(const float2 *__restrict__ z, int n, long long npix,
                                                      float *__restrict__ sum_pow, float *__restrict__ sum_amp,
                                                      int accumulate, const SumWeights wts) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
        float P = 0.0f, A = 0.0f;
        for (int t = 0; t < n; ++t) {
            const float2 v = __ldcs(z + (long long)t * npix + p);
            const float q = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
            P = __fadd_rn(P, __fmul_rn(wts.w[t], q));
            A = __fadd_rn(A, __fmul_rn(wts.w[t], __fsqrt_rn(q)));
        }
        if (accumulate) {
            P = __fadd_rn(__fmul_rn(wts.s, sum_pow[p]), P);
            if (sum_amp) A = __fadd_rn(__fmul_rn(wts.s, sum_amp[p]), A);
        }
        sum_pow[p] = P;
        if (sum_amp) sum_amp[p] = A;
    }
}

// One thread per output pixel; the window's power sums come through L1.
// Bit b = (dy+hy)*wx + (dx+hx); words are flushed as soon as they fill.
__global__ void __launch_bounds__(256) k_shp(const float *__restrict__ P, const Geom g, float c,
                                             uint64_t *__restrict__ mask, uint16_t *__restrict__ count) {
    const long long nout = (long long)g.Ho * g.Wo;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += stride) {
        const int i = (int)(o / g.Wo), j = (int)(o % g.Wo);
        const int cy = i * g.sy + g.sy / 2, cx = j * g.sx + g.sx / 2;
        const float Pp = __ldg(P + (long long)cy * g.W + cx);
        const bool valid = Pp > 0.0f;
        uint64_t cur = 0;
        int b = 0, w = 0, cnt = 0;
        uint64_t *m = mask + o * g.nwords;
        for (int dy = -g.hy; dy <= g.hy; ++dy) {
            const int y = cy + dy;
            const bool yin = (y >= 0) && (y < g.H);
            for (int dx = -g.hx; dx <= g.hx; ++dx, ++b) {
                const int x = cx + dx;
                bool acc = false;
                if (valid && yin && x >= 0 && x < g.W) {
                    const float Pq = __ldg(P + (long long)y * g.W + x);
                    const float hi = fmaxf(Pp, Pq), lo = fminf(Pp, Pq);
                    acc = (Pq > 0.0f) && (hi <= __fmul_rn(c, lo));
                }
                if (acc) {
                    cur |= 1ull << (b & 63);
                    ++cnt;
                }
                if ((b & 63) == 63) {
                    m[w++] = cur;
                    cur = 0;
                }
            }
        }
        if (b & 63) m[w] = cur;
        count[o] = (uint16_t)cnt;
    }
}

// Grid-stride launches: one full wave of resident blocks (or fewer if the
// work is smaller), so no partial second wave of equal-sized blocks.
static int grid_for(long long work, int block, int per_sm = 8) {
    const int sms = device_sm_count();
    long long blocks = (work + block - 1) / block;
    const long long cap = (long long)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <class K>
static int resident_per_sm(K kernel, int block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

cudaError_t launch_amp_stats(const float2 *z, int n, long long npix, float *sum_pow, float *sum_amp,
                             int accumulate, cudaStream_t s, const PsStats *ps, const SumWeights *wts) {
    if (npix == 0) return cudaSuccess;
    if (wts) {
        k_amp_stats_w<<<grid_for(npix, 256), 256, 0, s>>>(z, n, npix, sum_pow, sum_amp, accumulate, *wts);
    } else if (ps && ps->da && ps->amp_new && sum_amp) {
        static int per_sm = 0;  // per process: the kernel's residency does not change
        if (per_sm == 0) per_sm = std::min(8, resident_per_sm(k_amp_stats<true>, 256));
        k_amp_stats<true><<<grid_for(npix, 256, per_sm), 256, 0, s>>>(z, n, npix, sum_pow, sum_amp, accumulate,
                                                                      *ps);
    } else {
        k_amp_stats<false><<<grid_for(npix, 256), 256, 0, s>>>(z, n, npix, sum_pow, sum_amp, accumulate,
                                                               PsStats());
    }
    return cudaGetLastError();
}

cudaError_t launch_shp(const float *sum_pow, const Geom &g, float c, uint64_t *mask, uint16_t *count,
                       cudaStream_t s) {
    const long long nout = (long long)g.Ho * g.Wo;
    if (nout == 0) return cudaSuccess;
    k_shp<<<grid_for(nout, 256), 256, 0, s>>>(sum_pow, g, c, mask, count);
    return cudaGetLastError();
}

}  // namespace plk
