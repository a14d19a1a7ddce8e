// S7. Compressed SLC (Sec. II-B): kappa = zeta^H z over the real SLCs, each
// full-resolution pixel using the linked phases of the output cell whose
// decimation block contains it.  One thread per pixel; consecutive threads
// share a cell, so the phase loads hit L1.  HBM-streaming.
#include "plk_internal.cuh"

namespace plk {

__global__ void __launch_bounds__(256) k_compress(const __grid_constant__ Planes z, int n, int first_real,
                                                  const Geom g, const float *__restrict__ phase,
                                                  float2 *__restrict__ kappa) {
    const long long npix = (long long)g.H * g.W;
    const long long nout = (long long)g.Ho * g.Wo;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += stride) {
        const int y = (int)(q / g.W), x = (int)(q - (q / g.W) * g.W);
        const int ci = min(y / g.sy, g.Ho - 1), cj = min(x / g.sx, g.Wo - 1);
        const long long o = (long long)ci * g.Wo + cj;
        float kr = 0.f, ki = 0.f;
        bool bad = false;
        for (int i = first_real; i < n; ++i) {
            const float ph = __ldg(phase + (long long)i * nout + o);
            bad |= isnan(ph);
            float s, c;
            sincosf(ph, &s, &c);
            const float2 v = __ldcs(z.p[i] + q);
            // exp(-j ph) * v
            kr += c * v.x + s * v.y;
            ki += c * v.y - s * v.x;
        }
        kappa[q] = bad ? make_float2(0.f, 0.f) : make_float2(kr, ki);
    }
}

cudaError_t launch_compress(const Planes &z, int n, int first_real, const Geom &g, const float *phase,
                            float2 *kappa, cudaStream_t s) {
    const long long npix = (long long)g.H * g.W;
    if (npix == 0) return cudaSuccess;
    if (g.Ho == 0 || g.Wo == 0) return cudaMemsetAsync(kappa, 0, npix * sizeof(float2), s);
    long long blocks = (npix + 255) / 256;
    const long long cap = (long long)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_compress<<<(unsigned)blocks, 256, 0, s>>>(z, n, first_real, g, phase, kappa);
    return cudaGetLastError();
}

}  // namespace plk
