// Persistent-scatterer decision shared by the regridding and compression
// kernels (Sec. III-A, D_A = sigma_A / mu_A; Sec. IV, threshold on D_A).
#pragma once

#include "plk_internal.cuh"

namespace plk {

// With mu = SA / n and var = SP / n - mu^2 (eq. (merged-variance), one weight
// per image), D_A = sqrt(var) / mu = sqrt(max(n SP - SA^2, 0)) / SA, taken in
// that form: single precision, each operation correctly rounded in this order
// (no fused multiply-add), so any IEEE implementation of the same formula
// takes the same PS decisions.  Returns +inf where SA <= 0 (never a PS).
__device__ __forceinline__ float amp_dispersion(float sp, float sa, float n) {
    if (!(sa > 0.f)) return __int_as_float(0x7f800000);
    const float d = fmaxf(__fsub_rn(__fmul_rn(n, sp), __fmul_rn(sa, sa)), 0.f);
    return __fdiv_rn(__fsqrt_rn(d), sa);
}

// A PS's phases arg(z_i conj z_ref) must be defined: nonzero samples at the
// reference entry and on every real date.
__device__ __forceinline__ bool ps_samples_nonzero(const Planes &z, int n, int first_real, int ref, long long q) {
    float2 r = __ldg(z.p[ref] + q);
    if (r.x == 0.f && r.y == 0.f) return false;
    for (int i = first_real; i < n; ++i) {
        r = __ldg(z.p[i] + q);
        if (r.x == 0.f && r.y == 0.f) return false;
    }
    return true;
}

__device__ __forceinline__ bool ref_sample_nonzero(const Planes &z, int ref, long long q) {
    const float2 r = __ldg(z.p[ref] + q);
    return r.x != 0.f || r.y != 0.f;
}

}  // namespace plk
