// Complex 16-bit integer samples (interleaved re, im: the sample format of
// Sentinel-1 SLC products) widened to complex64, exactly (every int16 is a
// float).  HBM-bound: 4 bytes read and 8 written per sample; each thread moves
// four samples with one 16-byte load and two 16-byte stores.
#include "plk_internal.cuh"

namespace plk {

__global__ void k_ci16_to_c64(const int16_t *__restrict__ src, float2 *__restrict__ dst, long long n) {
    const long long n4 = n / 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const int4 v = __ldcs(s4 + i);  // streamed: read once
        float4 a, b;
        a.x = (float)(int16_t)(v.x & 0xffff);
        a.y = (float)(int16_t)((unsigned)v.x >> 16);
        a.z = (float)(int16_t)(v.y & 0xffff);
        a.w = (float)(int16_t)((unsigned)v.y >> 16);
        b.x = (float)(int16_t)(v.z & 0xffff);
        b.y = (float)(int16_t)((unsigned)v.z >> 16);
        b.z = (float)(int16_t)(v.w & 0xffff);
        b.w = (float)(int16_t)((unsigned)v.w >> 16);
        d4[2 * i] = a;
        d4[2 * i + 1] = b;
    }
    // the last n mod 4 samples
    const long long t = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = make_float2((float)src[2 * t], (float)src[2 * t + 1]);
}

cudaError_t launch_ci16_to_c64(const int16_t *src, float2 *dst, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long cap = (long long)device_sm_count() * 8;
    long long blocks = (n / 4 + 255) / 256;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    k_ci16_to_c64<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace plk
