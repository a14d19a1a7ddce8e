// Tensor-memory-accelerator (TMA) tile copies and mbarrier waits shared by the
// coherence kernels.  One 2D tensor map per date plane (elements of 8 bytes,
// i.e. one complex64 sample); a copy lands a box of RX x RY samples in shared
// memory and completes a transaction count on an mbarrier.  Every wait is
// bounded (about a second); a wait that gives up returns false and the caller
// raises its translation unit's timeout flag.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "plk_internal.cuh"

namespace plk {

struct TmaMaps {
    CUtensorMap m[PLK_MAX_N];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (about a second): false if the phase never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    for (int i = 0; i < (1 << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(256);
    }
    return false;
}
// Box copy to shared memory; x (the 8-byte-element column) must be even so
// that the copy starts on a 16-byte boundary.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on libcuda); null when unavailable.
static inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// One map per plane, box of bx x by samples (bx even).  False when TMA cannot
// serve the stack (W odd, a plane not 16-byte aligned, no encoder, a box
// dimension over 256, or an encoding error).
static inline bool encode_plane_maps(TmaMaps &maps, const Planes &z, int n, const Geom &g, int bx, int by) {
    if (g.W % 2 != 0 || bx > 256 || by > 256 || bx < 2 || by < 1 || tensor_map_encoder() == nullptr) return false;
    for (int d = 0; d < n; ++d)
        if (((uintptr_t)z.p[d] % 16) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)g.W, (cuuint64_t)g.H};
    const cuuint64_t strides[1] = {(cuuint64_t)g.W * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t estr[2] = {1, 1};
    for (int d = 0; d < n; ++d) {
        CUresult r = tensor_map_encoder()(&maps.m[d], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<float2 *>(z.p[d]),
                                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

}  // namespace plk
