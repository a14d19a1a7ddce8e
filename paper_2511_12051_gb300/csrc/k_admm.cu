// L1 time-series network inversion by ADMM (Sec. III-E, eq. (l1-min);
// Appendix): per pixel, minimise ||A x - b||_1 over the phase series x
// relative to the first date, b the unwrapped phases of the network's
// interferograms, by
//   x <- (A^T A)^{-1} A^T (b + z - u),  t = A x - b + u,
//   z <- S_{1/rho}(t),                  u <- t - z  (= clamp(t, -1/rho, 1/rho)),
// from z = u = 0, a fixed number of iterations.
//
// One thread per pixel: x, A^T v and u in registers, b in shared memory
// (column threadIdx.x of a [slot][128] array: every access of a warp is
// conflict-free); at most 128 registers a thread (4 CTAs an SM: with fewer
// registers the complete-network variant spills, and runs 28% slower).
// The networks are subsets of the nearest-3 network (pairs (a, a + d),
// d <= 3), so each pair has a compile-time slot admm_slot(NXP, d, a), NXP the
// number of unknown dates rounded up to an instantiated size: A x and A^T v
// are fixed register arithmetic, and A^T A is banded (bandwidth 3), its
// Cholesky factor L computed once on the host in double precision and passed
// in the parameter space; the solve is a banded forward and back substitution
// (4 FMA a row each way).  Slots the
// caller's network does not hold are skipped (a branch uniform across the
// grid), so they never reach x; for the complete nearest-3 network of the
// instantiated size there is no branch at all.  Each slot's b is read from the
// caller's interferogram plane by a uniform index (coalesced across the warp).
#include "plk_internal.cuh"

namespace plk {

constexpr int kAdmmThreads = 128;

// FULL: the network is every pair of the nearest-3 network over NXP unknown
// dates (no slot is masked, no branch); otherwise slots outside the network
// are skipped by a branch that is uniform across the grid.
template <int NXP, bool FULL>
__global__ void __launch_bounds__(kAdmmThreads, 4) k_admm_l1(const float *__restrict__ unw, long long npx,
                                                 const __grid_constant__ AdmmNet net, float *__restrict__ x_out) {
    constexpr int NS = 3 * NXP - 3;
    extern __shared__ float b_sh[];  // [NS][kAdmmThreads]
    float *b = b_sh + threadIdx.x;   // b[s * kAdmmThreads]: this thread's slot s
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npx; p += stride) {
        float u[NS], x[NXP], w[NXP];
        // v = b + z - u = b at the start
#pragma unroll
        for (int i = 0; i < NXP; ++i) w[i] = 0.f;
#pragma unroll
        for (int d = 1; d <= 3; ++d)
#pragma unroll
            for (int a = 0; a + d <= NXP; ++a) {
                const int s = admm_slot(NXP, d, a);
                const float bv = net.plane[s] >= 0 ? __ldg(unw + net.plane[s] * npx + p) : 0.f;
                b[s * kAdmmThreads] = bv;
                u[s] = 0.f;
                w[a + d - 1] += bv;
                if (a >= 1) w[a - 1] -= bv;
            }
        for (int it = 0; it < net.iters; ++it) {
            // x = (A^T A)^{-1} w: L y = w, then L^T x = y (L banded, stored by band).
#pragma unroll
            for (int i = 0; i < NXP; ++i) {
                float acc = w[i];
#pragma unroll
                for (int k = 1; k <= 3; ++k)
                    if (i - k >= 0) acc -= net.L[i][k] * x[i - k];
                x[i] = acc * net.L[i][0];
            }
#pragma unroll
            for (int i = NXP - 1; i >= 0; --i) {
                float acc = x[i];
#pragma unroll
                for (int k = 1; k <= 3; ++k)
                    if (i + k < NXP) acc -= net.L[i + k][k] * x[i + k];
                x[i] = acc * net.L[i][0];
            }
            // t = A x - b + u;  u = clamp(t);  v = b + z - u = b + t - 2u;  w = A^T v
#pragma unroll
            for (int i = 0; i < NXP; ++i) w[i] = 0.f;
#pragma unroll
            for (int d = 1; d <= 3; ++d)
#pragma unroll
                for (int a = 0; a + d <= NXP; ++a) {
                    const int s = admm_slot(NXP, d, a);
                    if (FULL || net.plane[s] >= 0) {
                        const float ax = x[a + d - 1] - (a >= 1 ? x[a - 1] : 0.f);
                        const float bs = b[s * kAdmmThreads];
                        const float t = ax - bs + u[s];
                        u[s] = fminf(fmaxf(t, -net.kappa), net.kappa);
                        const float v = bs + t - 2.f * u[s];
                        w[a + d - 1] += v;
                        if (a >= 1) w[a - 1] -= v;
                    }
                }
        }
#pragma unroll
        for (int i = 0; i < NXP; ++i)
            if (i < net.nx) x_out[i * npx + p] = x[i];
    }
}

// Residual b - A x of every interferogram, a separate streaming pass (kept out
// of the solve, whose register budget it would otherwise double).
__global__ void __launch_bounds__(256) k_admm_residual(const float *__restrict__ unw, long long npx,
                                                       const __grid_constant__ AdmmNet net,
                                                       const float *__restrict__ x, float *__restrict__ resid) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npx; p += stride) {
        for (int d = 1; d <= 3; ++d)
            for (int a = 0; a + d <= net.nxp; ++a) {
                const int s = admm_slot(net.nxp, d, a);
                if (net.plane[s] < 0) continue;  // uniform
                const float xb = a + d - 1 < net.nx ? __ldg(x + (long long)(a + d - 1) * npx + p) : 0.f;
                const float xa = a >= 1 ? __ldg(x + (long long)(a - 1) * npx + p) : 0.f;
                resid[net.plane[s] * npx + p] = __ldg(unw + net.plane[s] * npx + p) - (xb - xa);
            }
    }
}

cudaError_t launch_admm_l1(const float *unw, long long npx, const AdmmNet &net, float *x, float *resid,
                           cudaStream_t s) {
    if (npx == 0) return cudaSuccess;
    const long long want = (npx + kAdmmThreads - 1) / kAdmmThreads;
    bool full = true;
    for (int s = 0; s < 3 * net.nxp - 3; ++s) full = full && net.plane[s] >= 0;
    void (*kern)(const float *, long long, const AdmmNet, float *);
    switch (net.nxp) {
        case 4: kern = full ? k_admm_l1<4, true> : k_admm_l1<4, false>; break;
        case 8: kern = full ? k_admm_l1<8, true> : k_admm_l1<8, false>; break;
        case 12: kern = full ? k_admm_l1<12, true> : k_admm_l1<12, false>; break;
        case 14: kern = full ? k_admm_l1<14, true> : k_admm_l1<14, false>; break;
        case 15: kern = full ? k_admm_l1<15, true> : k_admm_l1<15, false>; break;
        case 16: kern = full ? k_admm_l1<16, true> : k_admm_l1<16, false>; break;
        default: return cudaErrorInvalidValue;
    }
    const size_t smem = (size_t)(3 * net.nxp - 3) * kAdmmThreads * sizeof(float);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdmmThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)device_sm_count() * per_sm;
    kern<<<(unsigned)(want < cap ? want : cap), kAdmmThreads, smem, s>>>(unw, npx, net, x);
    e = cudaGetLastError();
    if (e != cudaSuccess || !resid) return e;
    const long long rwant = (npx + 255) / 256, rcap = (long long)device_sm_count() * 8;
    k_admm_residual<<<(unsigned)(rwant < rcap ? rwant : rcap), 256, 0, s>>>(unw, npx, net, x, resid);
    return cudaGetLastError();
}

}  // namespace plk
