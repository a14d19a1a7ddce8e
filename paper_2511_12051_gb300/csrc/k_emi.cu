// S4-S6 kernel over packed coherences: one NP-lane group per pixel (32/NP
// pixels per warp), single-precision solve, and a double-precision re-solve of
// the same pixel, inside the same group, for pixels whose |C| is
// ill-conditioned (see emi.cuh).
#include "emi.cuh"

namespace plk {

// Row r of the packed Hermitian coherence of one pixel, read from global memory.
template <class T>
struct PackedRow {
    const float2 *Cp;  // pixel base
    int n, r;
    __device__ __forceinline__ cpx<T> operator()(int k) const {
        const bool up = r <= k;
        const float2 v = __ldg(Cp + (up ? packed_index(n, r, k) : packed_index(n, k, r)));
        return mk<T>((T)v.x, up ? (T)v.y : -(T)v.y);
    }
};

constexpr int kEmiWarps = 4;

// Single-precision pass: one NP-lane group per pixel.  Pixels the solve flags
// get status kPending and no other output.
template <int NP>
__global__ void __launch_bounds__(kEmiWarps * 32) k_emi32(const float2 *__restrict__ C, int n, long long npx,
                                                          int ref, const EmiParams prm,
                                                          float *__restrict__ phase, float *__restrict__ tcoh,
                                                          float *__restrict__ lam, uint8_t *__restrict__ status) {
    constexpr int G = 32 / NP;
    __shared__ __align__(16) cpx<float> sbuf[kEmiWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / NP, r = lane - grp * NP;
    const int glane0 = grp * NP;
    const unsigned gmask = (NP == 32) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    const long long step = (long long)gridDim.x * kEmiWarps * G;

    for (long long base = ((long long)blockIdx.x * kEmiWarps + warp) * G; base < npx; base += step) {
        const long long p = base + grp;
        const bool valid = p < npx;
        const float2 *Cpix = C + (valid ? p : 0) * nt;
        bool nan = false;
        if (valid && r < n) nan = isnan(__ldg(Cpix + packed_index(n, r, r)).x);
        nan = __any_sync(gmask, nan);
        if (valid && !nan) {
            PackedRow<float> ld{Cpix, n, r};
            const PixelResult res = emi_solve<NP, float>(ld, r, n, ref, prm, &sbuf[warp][glane0], gmask, glane0, false);
            if (res.flag) {
                if (r == 0) status[p] = (uint8_t)kPending;
            } else {
                if (r < n) phase[(long long)r * npx + p] = res.phase;
                if (r == 0) {
                    if (tcoh) tcoh[p] = res.tcoh;
                    if (lam) lam[p] = res.lam;
                    status[p] = (uint8_t)res.status;
                }
            }
        } else if (valid) {
            if (r < n) phase[(long long)r * npx + p] = __int_as_float(0x7fc00000);
            if (r == 0) {
                if (tcoh) tcoh[p] = __int_as_float(0x7fc00000);
                if (lam) lam[p] = __int_as_float(0x7fc00000);
                status[p] = PLK_PX_NODATA;
            }
        }
        __syncwarp();
    }
}

// Double-precision re-solve of the pixels left pending.  Each warp scans 32
// statuses at a time, ballots the pending ones and hands them out, one per
// NP-lane group, until the chunk is done.
template <int NP>
__global__ void __launch_bounds__(kEmiWarps * 32) k_emi64(const float2 *__restrict__ C, int n, long long npx,
                                                          int ref, const EmiParams prm,
                                                          float *__restrict__ phase, float *__restrict__ tcoh,
                                                          float *__restrict__ lam, uint8_t *__restrict__ status) {
    constexpr int G = 32 / NP;
    __shared__ __align__(16) cpx<double> sbuf[kEmiWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / NP, r = lane - grp * NP;
    const int glane0 = grp * NP;
    const unsigned gmask = (NP == 32) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    const long long step = (long long)gridDim.x * kEmiWarps * 32;

    for (long long base = ((long long)blockIdx.x * kEmiWarps + warp) * 32; base < npx; base += step) {
        const long long pl = base + lane;
        const bool pend = pl < npx && status[pl] == (uint8_t)kPending;
        unsigned bal = __ballot_sync(0xffffffffu, pend);
        while (bal) {
            int mine = -1;
#pragma unroll
            for (int gg = 0; gg < G; ++gg) {
                if (bal) {
                    const int b = __ffs(bal) - 1;
                    if (gg == grp) mine = b;
                    bal &= bal - 1u;
                }
            }
            if (mine >= 0) {
                const long long p = base + mine;
                PackedRow<double> ld{C + p * nt, n, r};
                const PixelResult res =
                    emi_solve<NP, double>(ld, r, n, ref, prm, &sbuf[warp][glane0], gmask, glane0, true);
                if (r < n) phase[(long long)r * npx + p] = res.phase;
                if (r == 0) {
                    if (tcoh) tcoh[p] = res.tcoh;
                    if (lam) lam[p] = res.lam;
                    status[p] = (uint8_t)res.status;
                }
            }
            __syncwarp();
        }
    }
}

template <int NP>
static cudaError_t run_emi(const float2 *C, int n, long long npx, int ref, const EmiParams &prm, float *phase,
                           float *tcoh, float *lam, uint8_t *status, cudaStream_t s, Prof *prof) {
    constexpr int G = 32 / NP;
    const long long cap = (long long)device_sm_count() * 16;
    long long blocks = ((npx + G - 1) / G + kEmiWarps - 1) / kEmiWarps;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    if (prof) prof->begin("phase_link_fp32", s);
    k_emi32<NP><<<(unsigned)blocks, kEmiWarps * 32, 0, s>>>(C, n, npx, ref, prm, phase, tcoh, lam, status);
    cudaError_t e = cudaGetLastError();
    if (prof) prof->end(s);
    if (e != cudaSuccess || !prm.fp64_resolve) return e;
    long long blocks64 = ((npx + 31) / 32 + kEmiWarps - 1) / kEmiWarps;
    blocks64 = blocks64 > cap ? cap : (blocks64 < 1 ? 1 : blocks64);
    if (prof) prof->begin("phase_link_fp64", s);
    k_emi64<NP><<<(unsigned)blocks64, kEmiWarps * 32, 0, s>>>(C, n, npx, ref, prm, phase, tcoh, lam, status);
    e = cudaGetLastError();
    if (prof) prof->end(s);
    return e;
}

cudaError_t launch_phase_link(const float2 *C, int n, long long npx, int ref, const EmiParams &prm,
                              float *phase, float *tcoh, float *lam, uint8_t *status, cudaStream_t s, Prof *prof) {
    if (npx == 0) return cudaSuccess;
    if (n <= 8) return run_emi<8>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof);
    if (n <= 16) return run_emi<16>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof);
    return run_emi<32>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof);
}

}  // namespace plk
