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

template <int NP>
__global__ void __launch_bounds__(kEmiWarps * 32) k_emi(const float2 *__restrict__ C, int n, long long npx,
                                                        int ref, const EmiParams prm,
                                                        float *__restrict__ phase, float *__restrict__ tcoh,
                                                        float *__restrict__ lam, uint8_t *__restrict__ status) {
    constexpr int G = 32 / NP;
    // One 16-byte slot per lane: room for a double-complex row per group.
    __shared__ __align__(16) cpx<double> sbuf[kEmiWarps][32];
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

        // No-data pixel: NaN coherence.
        bool nan = false;
        if (valid && r < n) {
            const float2 v = __ldg(Cpix + packed_index(n, r, r));
            nan = isnan(v.x);
        }
        nan = __any_sync(gmask, nan);
        const bool solve = valid && !nan;
        const int nn = solve ? n : 2;  // dummy 2x2 identity for idle groups

        PixelResult res;
        {
            cpx<float> *fbuf = reinterpret_cast<cpx<float> *>(&sbuf[warp][glane0]);
            PackedRow<float> ld{Cpix, nn, r};
            if (solve) {
                res = emi_solve<NP, float>(ld, r, nn, ref, prm, fbuf, gmask, glane0, false);
            } else {
                res.flag = false;
            }
        }
        if (solve && res.flag) {
            PackedRow<double> ld{Cpix, nn, r};
            res = emi_solve<NP, double>(ld, r, nn, ref, prm, &sbuf[warp][glane0], gmask, glane0, true);
        }
        __syncwarp();

        if (valid) {
            if (!solve) {
                if (r < n) phase[(long long)r * npx + p] = __int_as_float(0x7fc00000);
                if (r == 0) {
                    if (tcoh) tcoh[p] = __int_as_float(0x7fc00000);
                    if (lam) lam[p] = __int_as_float(0x7fc00000);
                    status[p] = PLK_PX_NODATA;
                }
            } else {
                if (r < n) phase[(long long)r * npx + p] = res.phase;
                if (r == 0) {
                    if (tcoh) tcoh[p] = res.tcoh;
                    if (lam) lam[p] = res.lam;
                    status[p] = (uint8_t)res.status;
                }
            }
        }
    }
}

template <int NP>
static cudaError_t run_emi(const float2 *C, int n, long long npx, int ref, const EmiParams &prm, float *phase,
                           float *tcoh, float *lam, uint8_t *status, cudaStream_t s) {
    constexpr int G = 32 / NP;
    const long long groups = (npx + G - 1) / G;
    long long blocks = (groups + kEmiWarps - 1) / kEmiWarps;
    const long long cap = (long long)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_emi<NP><<<(unsigned)blocks, kEmiWarps * 32, 0, s>>>(C, n, npx, ref, prm, phase, tcoh, lam, status);
    return cudaGetLastError();
}

cudaError_t launch_phase_link(const float2 *C, int n, long long npx, int ref, const EmiParams &prm,
                              float *phase, float *tcoh, float *lam, uint8_t *status, cudaStream_t s) {
    if (npx == 0) return cudaSuccess;
    if (n <= 8) return run_emi<8>(C, n, npx, ref, prm, phase, tcoh, lam, status, s);
    if (n <= 16) return run_emi<16>(C, n, npx, ref, prm, phase, tcoh, lam, status, s);
    return run_emi<32>(C, n, npx, ref, prm, phase, tcoh, lam, status, s);
}

}  // namespace plk
