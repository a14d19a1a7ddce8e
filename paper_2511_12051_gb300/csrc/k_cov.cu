// S3. SHP-windowed sample coherence (Sec. II-A, eq. (sample-coherence)).
//
// A CTA owns a TY x TX tile of output pixels.  It stages the input region the
// tile's windows cover (tile + halo, all N dates) in shared memory once, so
// each input sample is read from HBM about once per tile and the overlap of
// neighbouring windows is served from shared memory.
//
// The Hermitian sum S = sum_q z(q) z(q)^H is split into B x B register blocks
// over a BN x BN block grid; only the BN(BN+1)/2 upper blocks are computed.
// U = BN(BN+1)/2 lanes serve one output pixel, so a warp accumulates
// PPW = 32 / U pixels at once (5 pixels for N <= 18 with BN = 3).  Per window
// offset a lane loads 2B samples (broadcast within the pixel's lanes) and
// issues B*B complex multiply-adds; rejected looks contribute zero through a
// select, so every lane of the warp runs the same loop.
#include <algorithm>

#include "cpx.cuh"
#include "plk_internal.cuh"

namespace plk {

template <int BN>
__device__ __forceinline__ int diag_lane(int b) { return b * BN - b * (b - 1) / 2; }

template <int B, int BN>
__global__ void __launch_bounds__(128) k_cov(const __grid_constant__ Planes z, int n, const Geom g,
                                             const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                             int TY, int TX, int RY, int RX) {
    extern __shared__ float2 sm[];  // [n][RY][RX]
    constexpr int U = BN * (BN + 1) / 2;
    constexpr int PPW = 32 / U;
    const int tilesX = (g.Wo + TX - 1) / TX;
    const int ty0 = (int)(blockIdx.x / tilesX) * TY;
    const int tx0 = (int)(blockIdx.x % tilesX) * TX;
    const int y0 = ty0 * g.sy + g.sy / 2 - g.hy;
    const int x0 = tx0 * g.sx + g.sx / 2 - g.hx;
    const int plane = RY * RX;

    for (int idx = threadIdx.x; idx < n * plane; idx += blockDim.x) {
        const int d = idx / plane, rem = idx - d * plane;
        const int ry = rem / RX, rx = rem - ry * RX;
        const int y = y0 + ry, x = x0 + rx;
        float2 v = make_float2(0.f, 0.f);
        if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = __ldg(z.p[d] + (long long)y * g.W + x);
        sm[idx] = v;
    }
    __syncthreads();

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

    int offi[B], offk[B];
    bool vi[B], vk[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const int i = bi * B + r, k = bk * B + r;
        vi[r] = i < n;
        vk[r] = k < n;
        offi[r] = (vi[r] ? i : 0) * plane;
        offk[r] = (vk[r] ? k : 0) * plane;
    }

    for (int s0 = warp * PPW; s0 < npx_tile; s0 += nwarps * PPW) {
        const int s_raw = s0 + gslot;
        // Lanes without a pixel (idle lanes, slots past the tile) read slot 0's
        // window so every shared-memory address stays inside the staged region.
        const bool in_tile = lane_active && s_raw < npx_tile;
        const int s = in_tile ? s_raw : 0;
        const int ty = s / TX, tx = s - (s / TX) * TX;
        const int oy = ty0 + ty, ox = tx0 + tx;
        const bool pix_ok = in_tile && oy < g.Ho && ox < g.Wo;
        const long long o = (long long)oy * g.Wo + ox;
        const uint64_t *mw = mask + (pix_ok ? o : 0) * g.nwords;

        cpx<float> acc[B][B];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int q = 0; q < B; ++q) acc[r][q] = mk<float>(0.f, 0.f);

        const int cyr = ty * g.sy + g.hy, cxr = tx * g.sx + g.hx;
        uint64_t word = pix_ok ? __ldg(mw) : 0ull;
        int b = 0, L = 0;
        for (int dy = -g.hy; dy <= g.hy; ++dy) {
            const int rowoff = (cyr + dy) * RX + cxr;
            for (int dx = -g.hx; dx <= g.hx; ++dx, ++b) {
                if ((b & 63) == 0 && b > 0) word = pix_ok ? __ldg(mw + (b >> 6)) : 0ull;
                const bool on = (word >> (b & 63)) & 1ull;
                L += on;
                const int off = rowoff + dx;
                cpx<float> zi[B], zk[B];
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const float2 a = sm[offi[r] + off];
                    const float2 c = sm[offk[r] + off];
                    const bool ai = on && vi[r], ak = on && vk[r];
                    zi[r] = mk<float>(ai ? a.x : 0.f, ai ? a.y : 0.f);
                    zk[r] = mk<float>(ak ? c.x : 0.f, ak ? c.y : 0.f);
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

struct CovTile { int TY, TX, RY, RX; size_t smem; };

static CovTile choose_tile(int n, const Geom &g, int ppw, size_t budget) {
    CovTile best{0, 0, 0, 0, 0};
    double best_score = -1.0;
    const int per_pass = 4 * ppw;  // 4 warps per CTA
    for (int TY = 1; TY <= 16; ++TY)
        for (int TX = 1; TX <= 32; ++TX) {
            const int RY = (TY - 1) * g.sy + g.wy, RX = (TX - 1) * g.sx + g.wx;
            const size_t smem = (size_t)n * RY * RX * sizeof(float2);
            if (smem > budget) continue;
            const int px = TY * TX;
            if (px > 8 * per_pass) continue;
            const int passes = (px + per_pass - 1) / per_pass;
            const double lane_eff = (double)px / (passes * per_pass);
            const double halo_eff = (double)(TY * g.sy) * (TX * g.sx) / ((double)RY * RX);
            const double score = lane_eff * (0.5 + 0.5 * halo_eff) * (passes > 1 ? 1.0 : 0.98);
            if (score > best_score) {
                best_score = score;
                best = CovTile{TY, TX, RY, RX, smem};
            }
        }
    return best;
}

template <int B, int BN>
static cudaError_t run_cov(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                           cudaStream_t s) {
    constexpr int U = BN * (BN + 1) / 2;
    constexpr int PPW = 32 / U;
    CovTile t = choose_tile(n, g, PPW, 96 * 1024);
    if (t.TY == 0) t = choose_tile(n, g, PPW, 220 * 1024);
    if (t.TY == 0) return cudaErrorInvalidConfiguration;
    static int configured_max = 0;
    if ((int)t.smem > configured_max) {
        cudaError_t e = cudaFuncSetAttribute(k_cov<B, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e != cudaSuccess) return e;
        configured_max = 220 * 1024;
    }
    const long long tiles = (long long)((g.Ho + t.TY - 1) / t.TY) * ((g.Wo + t.TX - 1) / t.TX);
    if (tiles == 0) return cudaSuccess;
    k_cov<B, BN><<<(unsigned)tiles, 128, t.smem, s>>>(z, n, g, mask, C, t.TY, t.TX, t.RY, t.RX);
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
