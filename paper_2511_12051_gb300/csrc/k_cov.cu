// S3. SHP-windowed sample coherence (Sec. II-A, eq. (sample-coherence)).
//
// A CTA owns a TY x TX tile of output pixels and the input region their
// windows cover (tile + halo, all N date planes).  The Hermitian sum
// S = sum_q z(q) z(q)^H is split into B x B register blocks over a BN x BN
// block grid; only the BN(BN+1)/2 upper blocks are computed.  U = BN(BN+1)/2
// lanes serve one output pixel, so a warp accumulates PPW = 32/U pixels at
// once (5 pixels for N <= 18 with BN = 3).  Per window offset a lane loads 2B
// samples and issues B*B complex multiply-adds.  The SHP mask is applied by
// pointing the row-block loads of a rejected look at a zeroed pad pixel (one
// select per look), so every lane of the warp runs the same loop.
//
// Shared-memory layout for the compute: plane pitch PSc = 1 (mod 16 words of
// 8 bytes) and row pitch RXc with sy*RXc = 1 (mod 16); a warp's PPW pixels are
// stacked vertically, so one load instruction touches words
// (plane + row) mod 16 = (bi*B + r + ty) mod 16 -- distinct for B >= PPW and
// B*BN <= 16 -- and runs without bank conflicts.
//
// Staging: the TMA kernel (k_cov_tma) is persistent (one CTA per SM).  One
// thread issues one 2D tensor copy per date plane (cp.async.bulk.tensor, out-
// of-image parts zero-filled) into a 128-byte aligned staging buffer and
// signals an mbarrier; all threads re-lay the tile into the padded compute
// buffer, and the staging buffer immediately takes the next tile's copies
// while the warps compute.  Every mbarrier wait is bounded; a wait that gives
// up sets a device flag (read by plk_sync) and the CTA returns.
// k_cov_plain loads with ordinary coalesced loads (no alignment needs); it is
// used when a plane is not 16-byte aligned, W is odd or a box is too large.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "cpx.cuh"
#include "plk_internal.cuh"

namespace plk {

__device__ int g_wait_timeout = 0;

struct CovLayout {
    int TY, TX;    // output tile
    int RY, RX;    // staged region: rows, columns (columns start on an even image column)
    int RXc, PSc;  // compute buffer: row pitch, plane pitch (elements); zero pixel at RY*RXc
    int PSs;       // staging plane pitch (elements, multiple of 16 = 128 bytes)
    size_t smem_plain, smem_tma;
};

template <int BN>
__device__ __forceinline__ int diag_lane(int b) { return b * BN - b * (b - 1) / 2; }

// Accumulate, normalise and store the coherence of the tile's pixels from the
// compute buffer.  xoff: column of the region's first intended column.
template <int B, int BN>
__device__ __forceinline__ void cov_tile(const float2 *__restrict__ cmp, const int PSc, const int RXc, const int n,
                                         const Geom &g, const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                         const int ty0, const int tx0, const int TY, const int TX, const int RY,
                                         const int xoff) {
    constexpr int U = BN * (BN + 1) / 2;
    constexpr int PPW = 32 / U;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gslot = lane / U, u = lane - gslot * U;
    int bi = 0, bk = 0;
    {
        int t = u;
#pragma unroll
        for (int a = 0; a < BN; ++a) {
            const int len = BN - a;
            if (t >= 0 && t < len) { bi = a; bk = a + t; }
            t -= len;
        }
    }
    const bool lane_active = gslot < PPW;
    const int npx_tile = TY * TX;
    const int zoff = RY * RXc;  // the zero pixel of every compute plane

    int offi[B], offk[B];
    bool vi[B], vk[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const int i = bi * B + r, k = bk * B + r;
        vi[r] = i < n;
        vk[r] = k < n;
        offi[r] = (vi[r] ? i : 0) * PSc;
        offk[r] = (vk[r] ? k : 0) * PSc;
    }

    for (int s0 = warp * PPW; s0 < npx_tile; s0 += nwarps * PPW) {
        const int s_raw = s0 + gslot;
        // Lanes without a pixel read slot 0's window: every shared-memory
        // address stays inside the staged region.
        const bool in_tile = lane_active && s_raw < npx_tile;
        const int s = in_tile ? s_raw : 0;
        const int tx = s / TY, ty = s - (s / TY) * TY;  // slots run down a column
        const int oy = ty0 + ty, ox = tx0 + tx;
        const bool pix_ok = in_tile && oy < g.Ho && ox < g.Wo;
        const long long o = (long long)oy * g.Wo + ox;
        const uint64_t *mw = mask + (pix_ok ? o : 0) * g.nwords;

        cpx<float> acc[B][B];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int q = 0; q < B; ++q) acc[r][q] = mk<float>(0.f, 0.f);

        const int cyr = ty * g.sy + g.hy, cxr = tx * g.sx + g.hx + xoff;
        uint64_t word = pix_ok ? __ldg(mw) : 0ull;
        int b = 0, L = 0;
        for (int dy = -g.hy; dy <= g.hy; ++dy) {
            const int rowoff = (cyr + dy) * RXc + cxr;
            for (int dx = -g.hx; dx <= g.hx; ++dx, ++b) {
                if ((b & 63) == 0 && b > 0) word = pix_ok ? __ldg(mw + (b >> 6)) : 0ull;
                const bool on = (word >> (b & 63)) & 1ull;
                L += on;
                const int off = rowoff + dx;
                const int offz = on ? off : zoff;  // rejected look: the row block reads zeros
                cpx<float> zi[B], zk[B];
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const float2 a = cmp[offi[r] + offz];
                    const float2 c = cmp[offk[r] + off];
                    zi[r] = mk<float>(a.x, a.y);
                    zk[r] = mk<float>(c.x, c.y);
                }
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int q = 0; q < B; ++q) acc[r][q] = cfma_conj(zi[r], zk[q], acc[r][q]);
            }
        }

        // Diagonal powers S_ii live in the diagonal-block lanes of this pixel.
        const int src_i = gslot * U + diag_lane<BN>(bi);
        const int src_k = gslot * U + diag_lane<BN>(bk);
        float di[B], dk[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            const float v = acc[r][r].x;
            di[r] = __shfl_sync(0xffffffffu, v, src_i & 31);
            dk[r] = __shfl_sync(0xffffffffu, v, src_k & 31);
        }
        if (pix_ok) {
            float2 *Co = C + o * ntri(n);
#pragma unroll
            for (int r = 0; r < B; ++r)
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const int i = bi * B + r, k = bk * B + q;
                    if (i < n && k < n && (bi != bk || r <= q)) {
                        float2 v;
                        if (L == 0) {
                            v = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
                        } else if (i == k) {
                            v = make_float2(1.f, 0.f);
                        } else if (di[r] > 0.f && dk[q] > 0.f) {
                            const float sc = rsqrtf(di[r]) * rsqrtf(dk[q]);
                            v = make_float2(acc[r][q].x * sc, acc[r][q].y * sc);
                        } else {
                            v = make_float2(0.f, 0.f);
                        }
                        Co[packed_index(n, i, k)] = v;
                    }
                }
        }
    }
}

// ------------------------------------------------------------ plain loads

template <int B, int BN>
__global__ void __launch_bounds__(256) k_cov_plain(const __grid_constant__ Planes z, int n, const Geom g,
                                                   const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                                   const CovLayout lay) {
    extern __shared__ __align__(16) float2 sm[];  // n planes of PSc
    const int tilesY = (g.Ho + lay.TY - 1) / lay.TY;
    const int ty0 = (int)(blockIdx.x % tilesY) * lay.TY;
    const int tx0 = (int)(blockIdx.x / tilesY) * lay.TX;
    const int y0 = ty0 * g.sy + g.sy / 2 - g.hy;
    const int x0 = tx0 * g.sx + g.sx / 2 - g.hx;
    const int plane = lay.RY * lay.RX;
    for (int idx = threadIdx.x; idx < n * plane; idx += blockDim.x) {
        const int d = idx / plane, rem = idx - d * plane;
        const int ry = rem / lay.RX, rx = rem - ry * lay.RX;
        const int y = y0 + ry, x = x0 + rx;
        float2 v = make_float2(0.f, 0.f);
        if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = __ldg(z.p[d] + (long long)y * g.W + x);
        sm[d * lay.PSc + ry * lay.RXc + rx] = v;
    }
    for (int d = threadIdx.x; d < n; d += blockDim.x) sm[d * lay.PSc + lay.RY * lay.RXc] = make_float2(0.f, 0.f);
    __syncthreads();
    cov_tile<B, BN>(sm, lay.PSc, lay.RXc, n, g, mask, C, ty0, tx0, lay.TY, lay.TX, lay.RY, 0);
}

// --------------------------------------------------------------- TMA path

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
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

template <int B, int BN>
__global__ void __launch_bounds__(256, 1) k_cov_tma(const __grid_constant__ TmaMaps tm, int n, const Geom g,
                                                    const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                                    const CovLayout lay, long long ntiles, int tilesY) {
    extern __shared__ __align__(128) unsigned char smraw[];
    // Staging planes must start on 128-byte boundaries: align the base by hand
    // (the allocation carries 128 spare bytes).
    unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
    float2 *stg = reinterpret_cast<float2 *>(base);   // n planes of PSs (128-byte aligned)
    float2 *cmp = stg + (size_t)n * lay.PSs;          // n planes of PSc
    __shared__ __align__(8) uint64_t bar;
    const unsigned tx_bytes = (unsigned)(n * lay.RY * lay.RX * sizeof(float2));

    auto origin = [&](long long t, int &ty0, int &tx0, int &x0, int &y0, int &xoff) {
        ty0 = (int)(t % tilesY) * lay.TY;
        tx0 = (int)(t / tilesY) * lay.TX;
        y0 = ty0 * g.sy + g.sy / 2 - g.hy;
        const int xr = tx0 * g.sx + g.sx / 2 - g.hx;
        x0 = xr - (xr & 1);  // tensor copies start on an even column (16-byte rule)
        xoff = xr - x0;
    };
    auto issue = [&](long long t) {
        int ty0, tx0, x0, y0, xoff;
        origin(t, ty0, tx0, x0, y0, xoff);
        mbar_expect_tx(&bar, tx_bytes);
        for (int d = 0; d < n; ++d) tma_load_2d(stg + (size_t)d * lay.PSs, &tm.m[d], x0, y0, &bar);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int d = threadIdx.x; d < n; d += blockDim.x) cmp[(size_t)d * lay.PSc + lay.RY * lay.RXc] = make_float2(0.f, 0.f);
    __syncthreads();
    long long t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) issue(t);
    unsigned parity = 0;
    const int plane = lay.RY * lay.RX;
    for (; t < ntiles; t += gridDim.x) {
        if (!mbar_wait_bounded(&bar, parity)) {
            atomicOr(&g_wait_timeout, 1);
            return;
        }
        parity ^= 1u;
        for (int idx = threadIdx.x; idx < n * plane; idx += blockDim.x) {
            const int d = idx / plane, rem = idx - d * plane;
            const int ry = rem / lay.RX, rx = rem - ry * lay.RX;
            cmp[(size_t)d * lay.PSc + ry * lay.RXc + rx] = stg[(size_t)d * lay.PSs + rem];
        }
        __syncthreads();  // staging consumed, compute buffer ready
        const long long nt = t + gridDim.x;
        if (threadIdx.x == 0 && nt < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order the reads above before the copies
            issue(nt);
        }
        int ty0, tx0, x0, y0, xoff;
        origin(t, ty0, tx0, x0, y0, xoff);
        cov_tile<B, BN>(cmp, lay.PSc, lay.RXc, n, g, mask, C, ty0, tx0, lay.TY, lay.TX, lay.RY, xoff);
        __syncthreads();  // compute buffer free for the next tile
    }
}

// Diagnostic: one warp waits on an mbarrier that nothing will complete.  The
// bounded wait gives up after about a second and raises the timeout flag, which
// plk_sync turns into PLK_ETIMEOUT; the context stays usable.
__global__ void k_wait_selftest() {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0) && threadIdx.x == 0) atomicOr(&g_wait_timeout, 1);
}

cudaError_t launch_wait_selftest(cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>();
    return cudaGetLastError();
}

// ------------------------------------------------------------------- host

int read_and_clear_wait_timeout() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeout, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_wait_timeout, &zero, sizeof(int));
    }
    return v;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Row pitch >= rx with sy * pitch = 1 (mod 16) when sy is odd (else odd pitch).
static int row_pitch(int rx, int sy) {
    for (int p = rx; p < rx + 32; ++p) {
        if (sy % 2 == 1) {
            if ((sy * p) % 16 == 1) return p;
        } else if (p % 2 == 1) {
            return p;
        }
    }
    return rx;
}

static CovLayout make_layout(int n, const Geom &g, int TY, int TX) {
    CovLayout l{};
    l.TY = TY;
    l.TX = TX;
    l.RY = (TY - 1) * g.sy + g.wy;
    l.RX = round_up((TX - 1) * g.sx + g.wx + 1, 2);
    l.RXc = row_pitch(l.RX, g.sy);
    l.PSc = l.RY * l.RXc + 1;
    while (l.PSc % 16 != 1) ++l.PSc;
    l.PSs = round_up(l.RY * l.RX, 16);
    l.smem_plain = (size_t)n * l.PSc * sizeof(float2);
    l.smem_tma = (size_t)n * (l.PSs + l.PSc) * sizeof(float2) + 128;
    return l;
}

// Tile choice: PPW pixels stacked per warp column, 8 warps, several passes for
// small strides; the score favours little halo per output pixel.
static CovLayout choose_layout(int n, const Geom &g, int ppw, size_t budget, bool tma) {
    CovLayout best{};
    double best_score = -1.0;
    for (int a = 1; a <= 4; ++a)
        for (int TX = 1; TX <= 64; ++TX) {
            const int TY = ppw * a;
            const int px = TY * TX;
            if (px > 8 * ppw * 8) continue;
            CovLayout l = make_layout(n, g, TY, TX);
            const size_t sm = tma ? l.smem_tma : l.smem_plain;
            if (sm > budget || l.RX > 256 || l.RY > 256) continue;
            const double halo = (double)(TY * g.sy) * (TX * g.sx) / ((double)l.RY * l.RX);
            const int per_pass = 8 * ppw;
            const double lane_eff = (double)px / (((px + per_pass - 1) / per_pass) * per_pass);
            const double score = lane_eff * (0.6 + 0.4 * halo);
            if (score > best_score) {
                best_score = score;
                best = l;
            }
        }
    return best;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

template <int B, int BN>
static cudaError_t run_cov(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                           cudaStream_t s) {
    constexpr int U = BN * (BN + 1) / 2;
    constexpr int PPW = 32 / U;
    const size_t kMaxSmem = 220 * 1024;
    bool tma = (g.W % 2 == 0) && tensor_map_encoder() != nullptr;
    for (int d = 0; d < n && tma; ++d) tma = ((uintptr_t)z.p[d] % 16) == 0;
    CovLayout lay{};
    if (tma) {
        lay = choose_layout(n, g, PPW, kMaxSmem, true);
        tma = lay.TY > 0;
    }
    if (tma) {
        TmaMaps maps;
        const cuuint64_t dims[2] = {(cuuint64_t)g.W, (cuuint64_t)g.H};
        const cuuint64_t strides[1] = {(cuuint64_t)g.W * sizeof(float2)};
        const cuuint32_t box[2] = {(cuuint32_t)lay.RX, (cuuint32_t)lay.RY};
        const cuuint32_t estr[2] = {1, 1};
        for (int d = 0; d < n && tma; ++d) {
            CUresult r = tensor_map_encoder()(&maps.m[d], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2,
                                              const_cast<float2 *>(z.p[d]), dims, strides, box, estr,
                                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            tma = (r == CUDA_SUCCESS);
        }
        if (tma) {
            cudaError_t e = cudaFuncSetAttribute(k_cov_tma<B, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kMaxSmem);
            if (e != cudaSuccess) return e;
            const int tilesY = (g.Ho + lay.TY - 1) / lay.TY;
            const long long ntiles = (long long)tilesY * ((g.Wo + lay.TX - 1) / lay.TX);
            if (ntiles == 0) return cudaSuccess;
            const long long grid = std::min<long long>(ntiles, device_sm_count());
            k_cov_tma<B, BN><<<(unsigned)grid, 256, lay.smem_tma, s>>>(maps, n, g, mask, C, lay, ntiles, tilesY);
            return cudaGetLastError();
        }
    }
    lay = choose_layout(n, g, PPW, 96 * 1024, false);
    if (lay.TY == 0) lay = choose_layout(n, g, PPW, kMaxSmem, false);
    if (lay.TY == 0) {
        lay = make_layout(n, g, 1, 1);
        if (lay.smem_plain > kMaxSmem) return cudaErrorInvalidConfiguration;
    }
    cudaError_t e =
        cudaFuncSetAttribute(k_cov_plain<B, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((g.Ho + lay.TY - 1) / lay.TY) * ((g.Wo + lay.TX - 1) / lay.TX);
    if (tiles == 0) return cudaSuccess;
    k_cov_plain<B, BN><<<(unsigned)tiles, 256, lay.smem_plain, s>>>(z, n, g, mask, C, lay);
    return cudaGetLastError();
}

cudaError_t launch_covariance(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                              cudaStream_t s) {
    // 3 x 3 block grid (5 pixels per warp) up to N = 18; 5 x 5 (2 per warp) beyond.
    if (n <= 3) return run_cov<1, 3>(z, n, g, mask, C, s);
    if (n <= 6) return run_cov<2, 3>(z, n, g, mask, C, s);
    if (n <= 9) return run_cov<3, 3>(z, n, g, mask, C, s);
    if (n <= 12) return run_cov<4, 3>(z, n, g, mask, C, s);
    if (n <= 15) return run_cov<5, 3>(z, n, g, mask, C, s);
    if (n <= 18) return run_cov<6, 3>(z, n, g, mask, C, s);
    if (n <= 20) return run_cov<4, 5>(z, n, g, mask, C, s);
    if (n <= 25) return run_cov<5, 5>(z, n, g, mask, C, s);
    if (n <= 30) return run_cov<6, 5>(z, n, g, mask, C, s);
    return run_cov<7, 5>(z, n, g, mask, C, s);
}

}  // namespace plk
