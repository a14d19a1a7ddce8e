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
// Shared-memory layout for the compute: pixel-major, cmp[(row * RXc + col) * S
// + date] with an odd pixel stride S >= B*BN fixed at compile time, so a lane's
// B loads of a look are one base address plus immediate offsets.  The row
// pitch RXc is picked on the host by counting, for the lane pattern above, the
// 8-byte words that one half-warp's load sends to each of the 16 banks.  A
// rejected look reads one of 16 zero pixels, the one in the same bank as the
// look itself, so masks do not add bank traffic.  Lanes past the last pixel
// slot repeat the last slot's first lanes (same addresses, no extra traffic).
//
// Staging: the TMA kernel (k_cov_tma) is persistent (one CTA per SM).  One
// thread issues one 2D tensor copy per date plane (cp.async.bulk.tensor, out-
// of-image parts zero-filled) into a 128-byte aligned staging buffer and
// signals an mbarrier; all threads transpose the tile into the pixel-major
// compute buffer, and the staging buffer immediately takes the next tile's copies
// while the warps compute.  Every mbarrier wait is bounded; a wait that gives
// up sets a device flag (read by plk_sync) and the CTA returns.
// k_cov_plain loads with ordinary coalesced loads (no alignment needs); it is
// used when a plane is not 16-byte aligned, W is odd or a box is too large.
#include <algorithm>

#include "cpx.cuh"
#include "plk_internal.cuh"
#include "tma.cuh"

namespace plk {

__device__ int g_wait_timeout = 0;

struct CovLayout {
    int TY, TX;    // output tile
    int RY, RX;    // staged region: rows, columns (columns start on an even image column)
    int RXc;       // compute buffer row pitch (pixels)
    int Z0;        // first of the 16 zero pixels (multiple of 16); Z0 + 16 pixels in all
    int PSs;       // staging plane pitch (elements, multiple of 16 = 128 bytes)
    size_t smem_plain, smem_tma;
};

template <int BN>
__device__ __forceinline__ int diag_lane(int b) { return b * BN - b * (b - 1) / 2; }

// Pixel stride of the compute buffer: at least B*BN dates, odd, so that 16
// consecutive pixels of one date fall in 16 different 8-byte banks.
template <int B, int BN>
struct PixStride {
    static constexpr int value = (B * BN) % 2 ? B * BN : B * BN + 1;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// B consecutive complex samples from a 32-bit shared address, one 8-byte load
// each with an immediate offset.
template <int R>
__device__ __forceinline__ void lds_one(cpx<float> &v, uint32_t a) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(a), "n"(R * 8));
}
template <int B, int R = 0>
__device__ __forceinline__ void lds_row(cpx<float> (&v)[B], uint32_t a) {
    if constexpr (R < B) {
        lds_one<R>(v[R], a);
        lds_row<B, R + 1>(v, a);
    }
}

// Accumulate, normalise and store the coherence of the tile's pixels from the
// pixel-major compute buffer cmp[(row * RXc + col) * S + date].  xoff: column
// of the region's first intended column.
template <int B, int BN>
__device__ __forceinline__ void cov_tile(const float2 *__restrict__ cmp, const int RXc, const int Z0, const int n,
                                         const Geom &g, const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                         const int ty0, const int tx0, const int TY, const int TX, const int xoff) {
    constexpr int U = BN * (BN + 1) / 2;
    constexpr int PPW = 32 / U;
    constexpr int S = PixStride<B, BN>::value;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const bool lane_active = lane < PPW * U;
    // Lanes past the last pixel slot repeat the loads of the last slot's first
    // lanes (same addresses: broadcast, no extra bank traffic) and store nothing.
    const int gslot = lane_active ? lane / U : PPW - 1;
    const int u = lane_active ? lane - gslot * U : lane - PPW * U;
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
    const int npx_tile = TY * TX;
    // 32-bit shared addresses of date bi*B (row block) and bk*B (column
    // block) of pixel 0; a look adds pixel * S * 8 bytes, date r adds 8 r.
    const uint32_t base_i = smem_addr(cmp) + bi * B * 8, base_k = smem_addr(cmp) + bk * B * 8;

    for (int s0 = warp * PPW; s0 < npx_tile; s0 += nwarps * PPW) {
        const int s_raw = s0 + gslot;
        const bool in_tile = lane_active && s_raw < npx_tile;
        const int s = min(s_raw, npx_tile - 1);        // every address stays inside the region
        const int tx = s / TY, ty = s - (s / TY) * TY;  // slots run down a column
        const int oy = ty0 + ty, ox = tx0 + tx;
        const bool px_exists = oy < g.Ho && ox < g.Wo;
        const bool pix_ok = in_tile && px_exists;  // this lane stores
        const long long o = (long long)oy * g.Wo + ox;
        // Repeating lanes read the same mask as the lanes they repeat.
        const uint32_t *mw = reinterpret_cast<const uint32_t *>(mask + (px_exists ? o : 0) * g.nwords);

        cpx<float> acc[B][B];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int q = 0; q < B; ++q) acc[r][q] = mk<float>(0.f, 0.f);

        int L = 0;
        uint32_t m = 0;
        int b = 0;
        int off = ty * g.sy * RXc + tx * g.sx + xoff;  // window corner (dy = -hy, dx = -hx)
        for (int dy = 0; dy < g.wy; ++dy, off += RXc - g.wx) {
            for (int dx = 0; dx < g.wx; ++dx, ++off, ++b) {
                if ((b & 31) == 0) {
                    m = px_exists ? __ldg(mw + (b >> 5)) : 0u;
                    L += __popc(m);
                }
                const bool on = m & 1u;
                m >>= 1;
                // A rejected look reads the zero pixel in the same bank (Z0 is
                // a multiple of 16).
                const int offz = on ? off : (Z0 | (off & 15));
                const uint32_t ai = base_i + (uint32_t)offz * (S * 8), ak = base_k + (uint32_t)off * (S * 8);
                cpx<float> zi[B], zk[B];
                lds_row<B>(zi, ai);
                lds_row<B>(zk, ak);
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

// Zero the whole compute buffer (pad dates and the 16 zero pixels stay zero).
template <int S>
__device__ __forceinline__ void zero_compute(float2 *cmp, const CovLayout &lay) {
    const int total = (lay.Z0 + 16) * S;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) cmp[idx] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------ plain loads

template <int B, int BN>
__global__ void __launch_bounds__(256) k_cov_plain(const __grid_constant__ Planes z, int n, const Geom g,
                                                   const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                                   const CovLayout lay) {
    constexpr int S = PixStride<B, BN>::value;
    extern __shared__ __align__(16) float2 sm[];  // (Z0 + 16) pixels of S dates
    const int tilesY = (g.Ho + lay.TY - 1) / lay.TY;
    const int ty0 = (int)(blockIdx.x % tilesY) * lay.TY;
    const int tx0 = (int)(blockIdx.x / tilesY) * lay.TX;
    const int y0 = ty0 * g.sy + g.sy / 2 - g.hy;
    const int x0 = tx0 * g.sx + g.sx / 2 - g.hx;
    zero_compute<S>(sm, lay);
    __syncthreads();
    // Warp w fills rows (date d, row ry) w, w + nwarps, ...; lanes run along the row.
    const int nw = blockDim.x >> 5, ln = threadIdx.x & 31;
    for (int row = threadIdx.x >> 5; row < n * lay.RY; row += nw) {
        const int d = row / lay.RY, ry = row - d * lay.RY;
        const int y = y0 + ry;
        for (int rx = ln; rx < lay.RX; rx += 32) {
            const int x = x0 + rx;
            float2 v = make_float2(0.f, 0.f);
            if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = __ldg(z.p[d] + (long long)y * g.W + x);
            sm[(ry * lay.RXc + rx) * S + d] = v;
        }
    }
    __syncthreads();
    cov_tile<B, BN>(sm, lay.RXc, lay.Z0, n, g, mask, C, ty0, tx0, lay.TY, lay.TX, 0);
}

// --------------------------------------------------------------- TMA path

template <int B, int BN>
__global__ void __launch_bounds__(256, 1) k_cov_tma(const __grid_constant__ TmaMaps tm, int n, const Geom g,
                                                    const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                                    const CovLayout lay, long long ntiles, int tilesY) {
    constexpr int S = PixStride<B, BN>::value;
    extern __shared__ __align__(128) unsigned char smraw[];
    // Staging planes must start on 128-byte boundaries: align the base by hand
    // (the allocation carries 128 spare bytes).
    unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
    float2 *stg = reinterpret_cast<float2 *>(base);  // n planes of PSs (128-byte aligned)
    float2 *cmp = stg + (size_t)n * lay.PSs;         // (Z0 + 16) pixels of S dates
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
    zero_compute<S>(cmp, lay);
    __syncthreads();
    long long t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) issue(t);
    unsigned parity = 0;
    const int nrows = n * lay.RY, nw = blockDim.x >> 5, ln = threadIdx.x & 31;
    for (; t < ntiles; t += gridDim.x) {
        if (!mbar_wait_bounded(&bar, parity)) {
            atomicOr(&g_wait_timeout, 1);
            return;
        }
        parity ^= 1u;
        // Transpose staged rows (date d, row ry) into the pixel-major buffer.
        // Warp w takes rows w, w + nwarps, ...; four rows per pass, all loads
        // before the stores.  (d, ry) advance without divisions.
        {
            int dr[4], yr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int row = (threadIdx.x >> 5) + u * nw;
                dr[u] = row / lay.RY;
                yr[u] = row - dr[u] * lay.RY;
            }
            for (int row0 = threadIdx.x >> 5; row0 < nrows; row0 += 4 * nw) {
                float2 v[4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = row0 + u * nw < nrows;
                    const float2 *src = stg + (size_t)dr[u] * lay.PSs + yr[u] * lay.RX;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rx = ln + 32 * h;
                        v[u][h] = (ok && rx < lay.RX) ? src[rx] : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (row0 + u * nw >= nrows) continue;
                    const float2 *src = stg + (size_t)dr[u] * lay.PSs + yr[u] * lay.RX;
                    float2 *dst = cmp + (size_t)yr[u] * lay.RXc * S + dr[u];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rx = ln + 32 * h;
                        if (rx < lay.RX) dst[rx * S] = v[u][h];
                    }
                    for (int rx = ln + 64; rx < lay.RX; rx += 32) dst[rx * S] = src[rx];  // rows over 64 columns
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    yr[u] += 4 * nw;
                    while (yr[u] >= lay.RY) {
                        yr[u] -= lay.RY;
                        ++dr[u];
                    }
                }
            }
        }
        __syncthreads();  // staging consumed, compute buffer ready
        const long long nt = t + gridDim.x;
        if (threadIdx.x == 0 && nt < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order the reads above before the copies
            issue(nt);
        }
        int ty0, tx0, x0, y0, xoff;
        origin(t, ty0, tx0, x0, y0, xoff);
        cov_tile<B, BN>(cmp, lay.RXc, lay.Z0, n, g, mask, C, ty0, tx0, lay.TY, lay.TX, xoff);
        __syncthreads();  // compute buffer free for the next tile
    }
}

// ---------------------------------------------------------- async copies

// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (the
// source address is then not read but must still be a valid pointer).
__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Persistent kernel, two CTAs per SM: each CTA copies its tile's region
// straight into the pixel-major compute buffer with per-element asynchronous
// copies (no staging buffer, no transpose pass), waits for them and computes;
// while one CTA waits for its copies the other computes.
template <int B, int BN>
__global__ void __launch_bounds__(256, 2) k_cov_async(const __grid_constant__ Planes z, int n, const Geom g,
                                                      const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                                      const CovLayout lay, long long ntiles, int tilesY) {
    constexpr int S = PixStride<B, BN>::value;
    extern __shared__ __align__(16) float2 sm[];  // (Z0 + 16) pixels of S dates
    zero_compute<S>(sm, lay);
    __syncthreads();
    const int nrows = n * lay.RY, nw = blockDim.x >> 5, ln = threadIdx.x & 31;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty0 = (int)(t % tilesY) * lay.TY;
        const int tx0 = (int)(t / tilesY) * lay.TX;
        const int y0 = ty0 * g.sy + g.sy / 2 - g.hy;
        const int x0 = tx0 * g.sx + g.sx / 2 - g.hx;
        const bool x_inside = x0 >= 0 && x0 + lay.RX <= g.W;
        // Warp w copies rows (date d, row ry) w, w + nwarps, ...; (d, ry)
        // advance without divisions.
        int d = (threadIdx.x >> 5) / lay.RY, ry = (threadIdx.x >> 5) - d * lay.RY;
        for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
            const int y = y0 + ry;
            const bool y_inside = y >= 0 && y < g.H;
            const float2 *plane = z.p[d];
            const float2 *srow = plane + (long long)(y_inside ? y : 0) * g.W + x0;
            float2 *drow = sm + (size_t)ry * lay.RXc * S + d;
            if (y_inside && x_inside) {
                for (int rx = ln; rx < lay.RX; rx += 32) cp_async8(drow + rx * S, srow + rx, 8);
            } else {
                for (int rx = ln; rx < lay.RX; rx += 32) {
                    const int x = x0 + rx;
                    const bool ok = y_inside && x >= 0 && x < g.W;
                    cp_async8(drow + rx * S, ok ? srow + rx : plane, ok ? 8 : 0);
                }
            }
            ry += nw;
            while (ry >= lay.RY) {
                ry -= lay.RY;
                ++d;
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // every copy of the tile has landed
        cov_tile<B, BN>(sm, lay.RXc, lay.Z0, n, g, mask, C, ty0, tx0, lay.TY, lay.TX, 0);
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

// Shared-memory passes of one warp's two load instructions (row block and
// column block of a look) in the pixel-major buffer: per half-warp, the
// largest number of distinct 8-byte words that share one of 16 banks.  The
// lanes are laid out as in cov_tile; its PPW pixels sit sy * pitch pixels apart.
static int bank_passes(int B, int BN, int S, int sy, int pitch) {
    const int U = BN * (BN + 1) / 2, PPW = 32 / U;
    int lane_slot[32], lane_bi[32], lane_bk[32];
    for (int lane = 0; lane < 32; ++lane) {
        int gs = lane / U, u = lane - gs * U;
        if (gs >= PPW) {
            gs = PPW - 1;
            u = lane - PPW * U;
        }
        int bi = 0, bk = 0, t = u;
        for (int a = 0; a < BN; ++a) {
            const int len = BN - a;
            if (t >= 0 && t < len) { bi = a; bk = a + t; }
            t -= len;
        }
        lane_slot[lane] = gs;
        lane_bi[lane] = bi;
        lane_bk[lane] = bk;
    }
    int total = 0;
    for (int which = 0; which < 2; ++which)
        for (int half = 0; half < 2; ++half) {
            long long addr[16];
            int na = 0;
            for (int l = half * 16; l < half * 16 + 16; ++l) {
                const long long a =
                    (long long)lane_slot[l] * sy * pitch * S + (long long)(which ? lane_bk[l] : lane_bi[l]) * B;
                bool seen = false;
                for (int j = 0; j < na; ++j) seen = seen || addr[j] == a;
                if (!seen) addr[na++] = a;
            }
            int per_bank[16] = {0}, worst = 0;
            for (int j = 0; j < na; ++j) worst = std::max(worst, ++per_bank[addr[j] % 16]);
            total += worst;
        }
    return total;
}

// Smallest row pitch >= rx with the fewest bank passes.
static int row_pitch(int B, int BN, int S, int rx, int sy) {
    int best = rx, best_cost = 1 << 30;
    for (int p = rx; p < rx + 16; ++p) {
        const int c = bank_passes(B, BN, S, sy, p);
        if (c < best_cost) {
            best_cost = c;
            best = p;
        }
    }
    return best;
}

static CovLayout make_layout(int n, int B, int BN, int S, const Geom &g, int TY, int TX) {
    CovLayout l{};
    l.TY = TY;
    l.TX = TX;
    l.RY = (TY - 1) * g.sy + g.wy;
    l.RX = round_up((TX - 1) * g.sx + g.wx + 1, 2);
    l.RXc = row_pitch(B, BN, S, l.RX, g.sy);
    l.Z0 = round_up(l.RY * l.RXc, 16);
    l.PSs = round_up(l.RY * l.RX, 16);
    l.smem_plain = (size_t)(l.Z0 + 16) * S * sizeof(float2);
    l.smem_tma = (size_t)n * l.PSs * sizeof(float2) + l.smem_plain + 128;
    return l;
}

// Tile choice: PPW pixels stacked per warp column, 8 warps, several passes for
// small strides; the score favours full warps and little halo per output pixel.
static CovLayout choose_layout(int n, int B, int BN, int S, const Geom &g, size_t budget, bool tma) {
    const int ppw = 32 / (BN * (BN + 1) / 2);
    CovLayout best{};
    double best_score = -1.0;
    for (int a = 1; a <= 4; ++a)
        for (int TX = 1; TX <= 64; ++TX) {
            const int TY = ppw * a;
            const int px = TY * TX;
            if (px > 8 * ppw * 8) continue;
            CovLayout l = make_layout(n, B, BN, S, g, TY, TX);
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

// Block shape for n dates, as launch_covariance dispatches: B x B register
// blocks on a BN x BN grid.
static void block_shape(int n, int &B, int &BN) {
    BN = n <= 18 ? 3 : 5;
    B = (n + BN - 1) / BN;
    if (BN == 5 && B < 5) B = 5;  // 4-date blocks on a 5 x 5 grid collide in banks
}

int covariance_tile_candidates(int n, const Geom &g, int (*tiles)[2], int max) {
    int B, BN;
    block_shape(n, B, BN);
    const int S = (B * BN) % 2 ? B * BN : B * BN + 1;
    const int ppw = 32 / (BN * (BN + 1) / 2);
    const size_t kHalfSm = 113 * 1024;
    struct Cand {
        double score;
        int TY, TX;
    };
    Cand c[256];
    int nc = 0;
    for (int a = 1; a <= 4; ++a)
        for (int TX = 1; TX <= 64 && nc < 256; ++TX) {
            const int TY = ppw * a;
            const int px = TY * TX;
            if (px > 8 * ppw * 8) continue;
            CovLayout l = make_layout(n, B, BN, S, g, TY, TX);
            if (l.smem_plain > kHalfSm) continue;
            const double halo = (double)(TY * g.sy) * (TX * g.sx) / ((double)l.RY * l.RX);
            const int per_pass = 8 * ppw;
            const double lane_eff = (double)px / (((px + per_pass - 1) / per_pass) * per_pass);
            c[nc++] = {lane_eff * (0.6 + 0.4 * halo), TY, TX};
        }
    std::sort(c, c + nc, [](const Cand &x, const Cand &y) { return x.score > y.score; });
    const int m = std::min(nc, max);
    for (int i = 0; i < m; ++i) {
        tiles[i][0] = c[i].TY;
        tiles[i][1] = c[i].TX;
    }
    return m;
}

template <int B, int BN>
static cudaError_t run_cov(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                           cudaStream_t s, const Schedule *sch) {
    constexpr int S = PixStride<B, BN>::value;
    const size_t kMaxSmem = 226 * 1024;
#ifndef PLK_COV_NO_ASYNC
    {
        // Two CTAs per SM: each compute buffer within half the SM's shared
        // memory (less the per-CTA reservation).
        const size_t kHalfSm = 113 * 1024;
        CovLayout la{};
        if (sch && sch->cov_TY > 0 && sch->cov_TX > 0 && sch->cov_TY % (32 / (BN * (BN + 1) / 2)) == 0) {
            la = make_layout(n, B, BN, S, g, sch->cov_TY, sch->cov_TX);
            if (la.smem_plain > kHalfSm) la = CovLayout{};
        }
        if (la.TY == 0) la = choose_layout(n, B, BN, S, g, kHalfSm, false);
        if (la.TY > 0) {
            cudaError_t e = cudaFuncSetAttribute(k_cov_async<B, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kHalfSm);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cov_async<B, BN>, 256, la.smem_plain);
            if (e != cudaSuccess) return e;
            if (per_sm >= 1) {
                const int tilesY = (g.Ho + la.TY - 1) / la.TY;
                const long long ntiles = (long long)tilesY * ((g.Wo + la.TX - 1) / la.TX);
                if (ntiles == 0) return cudaSuccess;
                const long long grid = std::min<long long>(ntiles, (long long)per_sm * device_sm_count());
                k_cov_async<B, BN><<<(unsigned)grid, 256, la.smem_plain, s>>>(z, n, g, mask, C, la, ntiles, tilesY);
                return cudaGetLastError();
            }
        }
    }
#endif
    CovLayout lay = choose_layout(n, B, BN, S, g, kMaxSmem, true);
    TmaMaps maps;
    if (lay.TY > 0 && encode_plane_maps(maps, z, n, g, lay.RX, lay.RY)) {
        cudaError_t e =
            cudaFuncSetAttribute(k_cov_tma<B, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (e != cudaSuccess) return e;
        const int tilesY = (g.Ho + lay.TY - 1) / lay.TY;
        const long long ntiles = (long long)tilesY * ((g.Wo + lay.TX - 1) / lay.TX);
        if (ntiles == 0) return cudaSuccess;
        const long long grid = std::min<long long>(ntiles, device_sm_count());
        k_cov_tma<B, BN><<<(unsigned)grid, 256, lay.smem_tma, s>>>(maps, n, g, mask, C, lay, ntiles, tilesY);
        return cudaGetLastError();
    }
    lay = choose_layout(n, B, BN, S, g, 96 * 1024, false);
    if (lay.TY == 0) lay = choose_layout(n, B, BN, S, g, kMaxSmem, false);
    if (lay.TY == 0) {
        lay = make_layout(n, B, BN, S, g, 1, 1);
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
                              cudaStream_t s, int precision, const Schedule *sch) {
    if (precision == 1) return launch_covariance_bf16(z, n, g, mask, C, s);
    if (precision == 2) return launch_covariance_fp16(z, n, g, mask, C, s);
    // 3 x 3 block grid (5 pixels per warp) up to N = 18; 5 x 5 (2 per warp) beyond
    // (blocks of 5 or more dates: 4-date blocks on a 5 x 5 grid collide in banks).
    // Kept in step with block_shape().
    if (n <= 3) return run_cov<1, 3>(z, n, g, mask, C, s, sch);
    if (n <= 6) return run_cov<2, 3>(z, n, g, mask, C, s, sch);
    if (n <= 9) return run_cov<3, 3>(z, n, g, mask, C, s, sch);
    if (n <= 12) return run_cov<4, 3>(z, n, g, mask, C, s, sch);
    if (n <= 15) return run_cov<5, 3>(z, n, g, mask, C, s, sch);
    if (n <= 18) return run_cov<6, 3>(z, n, g, mask, C, s, sch);
    if (n <= 25) return run_cov<5, 5>(z, n, g, mask, C, s, sch);
    if (n <= 30) return run_cov<6, 5>(z, n, g, mask, C, s, sch);
    return run_cov<7, 5>(z, n, g, mask, C, s, sch);
}

}  // namespace plk
