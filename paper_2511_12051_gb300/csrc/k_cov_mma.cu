// S3 in reduced precision: SHP-windowed sample coherence (Sec. II-A, eq.
// (sample-coherence)) with the samples rounded to bfloat16 or to half
// precision and the sums accumulated in single precision on the tensor cores
// (mma.sync m16n8k16).
//
// Half precision has three more significand bits than bfloat16 but a narrow
// exponent range, so each tile's samples are first scaled by one power of two
// that puts the tile's largest component in [2^14, 2^15): exact, and exactly
// cancelled by the normalisation C_ik = S_ik / sqrt(S_ii S_kk), since every
// window of the tile's output pixels lies inside the tile's region.
//
// Per output pixel the sum S = sum_q m(q) z(q) z(q)^H is a small dense
// contraction over its looks.  With x = Re z, y = Im z (vectors over dates)
// and the looks' (x, y) interleaved along the contraction index k:
//     Re S = Zr M Zr^T,   Im S = Zs M Zr^T,
// Zr[date][2l] = x_l, Zr[date][2l+1] = y_l;  Zs[date][2l] = y_l, Zs[date][2l+1] = -x_l,
// M the 0/1 mask (M = M^2, so it is applied to both factors by reading a zero
// pixel for a rejected look).
//
// Shared memory holds the tile's input region pixel-major: each pixel is a
// record of 16-byte units [x dates 0-7][y dates 0-7][x dates 8-15][y 8-15]...
// plus two pad units, so that the 8 rows of one 8x8 ldmatrix (4 consecutive
// looks x 2 components) fall in 8 different 16-byte bank groups.  One
// ldmatrix.x4.trans per 16 dates and 8 looks gives, in the same registers, the
// A fragments (dates x k) and the B fragments (k x dates) of both output
// column tiles; the Im product uses A' = (y, -x) formed from them by a half
// swap and a sign flip.  A warp owns one output pixel at a time; its lanes
// supply the row addresses, i.e. the window gather and the mask are free.
// Rows of rejected looks point at one of four zero pixels with the same bank
// position.
//
// The records are filled with ordinary coalesced loads (16 in flight per
// thread), rounded to 16 bits (round to nearest even) and stored with 16-byte
// stores; for N <= 16 two CTAs share an SM, one loading while the other runs
// its tensor work.  (A variant staging the region through TMA boxes, one CTA
// per SM, and one interleaving two pixels per warp were both slower.)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "plk_internal.cuh"

namespace plk {

namespace {

struct MmaLayout {
    int TY, TX;  // output tile
    int RY, RX;  // input region
    int Z0;      // first of 4 zero pixels (multiple of 4)
    int L;       // looks per window
    size_t smem;
};

template <int NT>
struct Rec {
    static constexpr int units = NT / 8 * 2 + 2;  // 16-byte units per pixel record
    static constexpr int bytes = units * 16;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// D += A B, m16n8k16, bfloat16 (F16 = false) or half-precision (F16 = true)
// inputs, single-precision accumulators.
template <bool F16>
__device__ __forceinline__ void mma_16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (F16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// (x, y) packed as (low, high) 16-bit values -> (y, -x) (the sign is bit 15
// of each half in both formats).
__device__ __forceinline__ uint32_t swap_neg(uint32_t v) { return __byte_perm(v, 0, 0x1032) ^ 0x80000000u; }

template <bool F16>
__device__ __forceinline__ uint32_t pack_16(float lo, float hi) {
    uint32_t u;
    if constexpr (F16) {
        const __half2 h = __floats2half2_rn(lo, hi);
        memcpy(&u, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        memcpy(&u, &h, 4);
    }
    return u;
}

// Store 8 samples (times the tile's scale) of one date group of one pixel as
// two units of 16-bit values.
template <bool F16>
__device__ __forceinline__ void store_group(unsigned char *rec, int q, const float2 (&v)[8], float sc) {
    uint4 ux, uy;
    ux.x = pack_16<F16>(v[0].x * sc, v[1].x * sc);
    ux.y = pack_16<F16>(v[2].x * sc, v[3].x * sc);
    ux.z = pack_16<F16>(v[4].x * sc, v[5].x * sc);
    ux.w = pack_16<F16>(v[6].x * sc, v[7].x * sc);
    uy.x = pack_16<F16>(v[0].y * sc, v[1].y * sc);
    uy.y = pack_16<F16>(v[2].y * sc, v[3].y * sc);
    uy.z = pack_16<F16>(v[4].y * sc, v[5].y * sc);
    uy.w = pack_16<F16>(v[6].y * sc, v[7].y * sc);
    uint4 *u = reinterpret_cast<uint4 *>(rec);
    u[2 * q] = ux;
    u[2 * q + 1] = uy;
}

// Shared-memory tables after the records: look offsets, per-warp staging of
// one pixel's packed output, per-warp diagonal.
template <int NT>
struct MmaSmem {
    unsigned char *rec;  // (Z0 + 4) records
    int *lkoff;          // L
    float2 *stage;       // 8 warps x NT(NT+1)/2
    float *diag;         // 8 warps x NT
    __device__ MmaSmem(unsigned char *base, const MmaLayout &lay) {
        rec = base;
        lkoff = reinterpret_cast<int *>(base + (size_t)(lay.Z0 + 4) * Rec<NT>::bytes);
        stage = reinterpret_cast<float2 *>(lkoff + ((lay.L + 3) & ~3));
        diag = reinterpret_cast<float *>(stage + (size_t)8 * (NT * (NT + 1) / 2));
    }
};

// Zero pixels and the window's look offsets (pixels, relative to the window
// corner): look l = dy * wx + dx, the SHP mask bit order.
template <int NT>
__device__ __forceinline__ void init_tables(const MmaSmem<NT> &s, const MmaLayout &lay, const Geom &g) {
    constexpr int PXB = Rec<NT>::bytes;
    for (int i = threadIdx.x; i < 4 * PXB / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(s.rec + (size_t)lay.Z0 * PXB)[i] = make_uint4(0, 0, 0, 0);
    for (int l = threadIdx.x; l < lay.L; l += blockDim.x) s.lkoff[l] = (l / g.wx) * lay.RX + (l % g.wx);
}

// Lane-constant roles: ldmatrix row (matrix m = lane / 8: k half m / 2, date
// half m % 2; row = lane % 8 -> k = (m / 2) * 8 + row) and the accumulator
// slots it owns (element e of tile (a, c): row 16a + g4 + 8 (e >> 1), column
// 8c + 2 t4 + (e & 1); slot bit (a * 2MT + c) * 4 + e).
template <int NT>
struct MmaLane {
    static constexpr int MT = NT / 16;
    int look_in_step, g4, t4;
    uint32_t unit_off, valid_bits, diag_bits;
    int rowbase[MT][2];  // i n - i(i-1)/2 - i of this lane's rows
    __device__ MmaLane(int n) {
        const int lane = threadIdx.x & 31;
        const int mtx = lane >> 3, row = lane & 7;
        const int kl = (mtx >> 1) * 8 + row;
        look_in_step = kl >> 1;
        unit_off = (uint32_t)((2 * (mtx & 1) + (kl & 1)) * 16);  // + 64 bytes per further 16 dates
        g4 = lane >> 2;
        t4 = lane & 3;
        valid_bits = diag_bits = 0;
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = 16 * a + g4 + 8 * h;
                rowbase[a][h] = i * n - i * (i - 1) / 2 - i;
            }
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int c = 0; c < 2 * MT; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = 16 * a + g4 + 8 * (e >> 1), kk = 8 * c + 2 * t4 + (e & 1);
                    const int bit = (a * 2 * MT + c) * 4 + e;
                    if (i <= kk && kk < n) valid_bits |= 1u << bit;
                    if (i == kk) diag_bits |= 1u << bit;
                }
    }
};

// Tensor-core sums, normalisation and packed stores for the tile's pixels,
// one pixel per warp at a time.
template <int NT, bool F16>
__device__ __forceinline__ void mma_tile(const MmaLane<NT> &ln, const MmaSmem<NT> &s, const MmaLayout &lay, int n,
                                         const Geom &g, const uint64_t *__restrict__ mask, float2 *__restrict__ C,
                                         int ty0, int tx0) {
    constexpr int MT = NT / 16;
    constexpr int PXB = Rec<NT>::bytes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nt = n * (n + 1) / 2;
    const int nsteps = (lay.L + 7) / 8;
    const uint32_t region_base = smem_u32(s.rec);
    const int npx_tile = lay.TY * lay.TX;
    for (int sl = warp; sl < npx_tile; sl += nwarps) {
        const int tx = sl / lay.TY, ty = sl - tx * lay.TY;
        const int oy = ty0 + ty, ox = tx0 + tx;
        const bool px_exists = oy < g.Ho && ox < g.Wo;
        const long long o = px_exists ? (long long)oy * g.Wo + ox : 0;
        const uint32_t *mw = reinterpret_cast<const uint32_t *>(mask + o * g.nwords);
        const int corner = ty * g.sy * lay.RX + tx * g.sx;
        float dre[MT][2 * MT][4], dim[MT][2 * MT][4];
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int b = 0; b < 2 * MT; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) dre[a][b][e] = dim[a][b][e] = 0.f;
        int L = 0;
        for (int w = 0; w * 32 < lay.L; ++w) L += px_exists ? __popc(__ldg(mw + w)) : 0;
        // Windows of up to 64 looks keep their mask in two registers.
        const uint32_t m0 = (px_exists && lay.L <= 64) ? __ldg(mw) : 0u;
        const uint32_t m1 = (px_exists && lay.L > 32 && lay.L <= 64) ? __ldg(mw + 1) : 0u;
        auto row_addr = [&](int step) {
            const int l = step * 8 + ln.look_in_step;
            bool on = false;
            int P = 0;
            if (l < lay.L) {
                P = corner + s.lkoff[l];
                const uint32_t w = lay.L <= 64 ? (l < 32 ? m0 : m1) : (px_exists ? __ldg(mw + (l >> 5)) : 0u);
                on = (w >> (l & 31)) & 1u;
            }
            const int Pz = on ? P : (lay.Z0 + (P & 3));
            return region_base + (uint32_t)Pz * PXB + ln.unit_off;
        };
        uint32_t f[MT][4];
        {
            const uint32_t a0 = row_addr(0);
#pragma unroll
            for (int a = 0; a < MT; ++a) ldsm_x4_trans(f[a], a0 + a * 64);
        }
        for (int step = 0; step < nsteps; ++step) {
            // Next step's fragments first: the loads overlap this step's MMAs.
            uint32_t fn[MT][4];
            if (step + 1 < nsteps) {
                const uint32_t an = row_addr(step + 1);
#pragma unroll
                for (int a = 0; a < MT; ++a) ldsm_x4_trans(fn[a], an + a * 64);
            }
            // f[a] = {dates 16a+0-7 k 0-7, dates 16a+8-15 k 0-7, dates 16a+0-7 k 8-15, dates 16a+8-15 k 8-15}
#pragma unroll
            for (int a = 0; a < MT; ++a) {
                uint32_t as[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) as[e] = swap_neg(f[a][e]);
#pragma unroll
                for (int b = 0; b < MT; ++b) {
                    // column tiles of 8 dates: 16b + 0-7 and 16b + 8-15
                    mma_16<F16>(dre[a][2 * b], f[a], f[b][0], f[b][2]);
                    mma_16<F16>(dre[a][2 * b + 1], f[a], f[b][1], f[b][3]);
                    mma_16<F16>(dim[a][2 * b], as, f[b][0], f[b][2]);
                    mma_16<F16>(dim[a][2 * b + 1], as, f[b][1], f[b][3]);
                }
            }
            if (step + 1 < nsteps) {
#pragma unroll
                for (int a = 0; a < MT; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e) f[a][e] = fn[a][e];
            }
        }

        float *dg = s.diag + warp * NT;
        __syncwarp();
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int c = 0; c < 2 * MT; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((ln.diag_bits >> ((a * 2 * MT + c) * 4 + e)) & 1u) dg[16 * a + ln.g4 + 8 * (e >> 1)] = dre[a][c][e];
        __syncwarp();
        // s_i = 1/sqrt(S_ii) for this lane's rows and columns (0 where S_ii = 0).
        float rr[MT][2], rc[2 * MT][2];
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float d = dg[16 * a + ln.g4 + 8 * h];
                rr[a][h] = d > 0.f ? rsqrtf(d) : 0.f;
            }
#pragma unroll
        for (int c = 0; c < 2 * MT; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float d = dg[8 * c + 2 * ln.t4 + j];
                rc[c][j] = d > 0.f ? rsqrtf(d) : 0.f;
            }
        float2 *st = s.stage + (size_t)warp * (NT * (NT + 1) / 2);
        const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int c = 0; c < 2 * MT; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int bit = (a * 2 * MT + c) * 4 + e;
                    if ((ln.valid_bits >> bit) & 1u) {
                        const float sc = rr[a][e >> 1] * rc[c][e & 1];
                        const bool dia = (ln.diag_bits >> bit) & 1u;
                        float2 v = dia ? make_float2(1.f, 0.f) : make_float2(dre[a][c][e] * sc, dim[a][c][e] * sc);
                        if (L == 0) v = make_float2(qnan, qnan);
                        st[ln.rowbase[a][e >> 1] + 8 * c + 2 * ln.t4 + (e & 1)] = v;
                    }
                }
        __syncwarp();
        if (px_exists) {
            float2 *Co = C + o * nt;
            for (int j = lane; j < nt; j += 32) Co[j] = st[j];
        }
        __syncwarp();
    }
}

}  // namespace

// Ordinary loads.  NT = 16 or 32 dates per pixel record (N <= NT).
template <int NT, bool F16>
__global__ void __launch_bounds__(256, NT == 16 ? 2 : 1) k_cov_mma(const __grid_constant__ Planes z, int n,
                                                                   const Geom g, const uint64_t *__restrict__ mask,
                                                                   float2 *__restrict__ C, const MmaLayout lay,
                                                                   long long ntiles, int tilesY) {
    constexpr int PXB = Rec<NT>::bytes;
    extern __shared__ __align__(16) unsigned char sm[];
    const MmaSmem<NT> s(sm, lay);
    init_tables<NT>(s, lay, g);
    const MmaLane<NT> ln(n);
    const int npx_region = lay.RY * lay.RX;
    // Load cursors of this thread's two tasks per pass (task = date group q,
    // pixel p = ry * RX + rx), advanced without divisions.
    const int ntask = (NT / 8) * npx_region;
    int cq[2], cy[2], cx[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int idx = threadIdx.x + h * blockDim.x;
        cq[h] = idx / npx_region;
        const int p = idx - cq[h] * npx_region;
        cy[h] = p / lay.RX;
        cx[h] = p - cy[h] * lay.RX;
    }
    const int adv = 2 * blockDim.x, adv_y = adv / lay.RX, adv_x = adv - adv_y * lay.RX;

    __shared__ unsigned tile_max;  // largest |component| of the region, as float bits (half precision only)
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty0 = (int)(t % tilesY) * lay.TY;
        const int tx0 = (int)(t / tilesY) * lay.TX;
        const int y0 = ty0 * g.sy + g.sy / 2 - g.hy;
        const int x0 = tx0 * g.sx + g.sx / 2 - g.hx;
        if (F16 && threadIdx.x == 0) tile_max = 0u;
        __syncthreads();  // previous tile's reads done (and the tables written)
        // One pass over this thread's tasks of the region: fn(h, v, ry, rx, q)
        // gets each task's 8 samples (zero outside the image and past n).
        auto for_tasks = [&](auto &&fn) {
            int q[2] = {cq[0], cq[1]}, ry[2] = {cy[0], cy[1]}, rx[2] = {cx[0], cx[1]};
            for (int idx0 = threadIdx.x; idx0 < ntask; idx0 += adv) {
                float2 v[2][8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int y = y0 + ry[h], x = x0 + rx[h];
                    const bool inside =
                        idx0 + h * (int)blockDim.x < ntask && y >= 0 && y < g.H && x >= 0 && x < g.W;
                    const long long off = inside ? (long long)y * g.W + x : 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int d = q[h] * 8 + u;
                        v[h][u] = (inside && d < n) ? __ldg(z.p[d] + off) : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (idx0 + h * (int)blockDim.x < ntask) fn(v[h], ry[h], rx[h], q[h]);
                    rx[h] += adv_x;
                    ry[h] += adv_y;
                    if (rx[h] >= lay.RX) {
                        rx[h] -= lay.RX;
                        ++ry[h];
                    }
                    while (ry[h] >= lay.RY) {
                        ry[h] -= lay.RY;
                        ++q[h];
                    }
                }
            }
        };
        float sc = 1.f;
        if constexpr (F16) {
            float m = 0.f;
            for_tasks([&](const float2 (&v)[8], int, int, int) {
#pragma unroll
                for (int u = 0; u < 8; ++u) m = fmaxf(m, fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
            });
            atomicMax(&tile_max, __float_as_uint(m));  // non-negative floats order as their bits
            __syncthreads();
            const float mx = __uint_as_float(tile_max);
            // 2^(14 - e) for mx in [2^e, 2^(e+1)): the largest component lands in [2^14, 2^15)
            if (mx > 0.f && mx < __int_as_float(0x7f800000)) sc = ldexpf(1.f, max(-126, min(127, 14 - ilogbf(mx))));
        }
        for_tasks([&](const float2 (&v)[8], int ry, int rx, int q) {
            store_group<F16>(s.rec + (size_t)(ry * lay.RX + rx) * PXB, q, v, sc);
        });
        __syncthreads();
        mma_tile<NT, F16>(ln, s, lay, n, g, mask, C, ty0, tx0);
    }
}

static int round_up_i(int v, int m) { return (v + m - 1) / m * m; }

static MmaLayout mma_layout(int NT, const Geom &g, int TY, int TX) {
    MmaLayout l{};
    l.TY = TY;
    l.TX = TX;
    l.RY = (TY - 1) * g.sy + g.wy;
    l.RX = (TX - 1) * g.sx + g.wx;
    l.Z0 = round_up_i(l.RY * l.RX, 4);
    l.L = g.wy * g.wx;
    const int rec = NT / 8 * 32 + 32;
    l.smem = (size_t)(l.Z0 + 4) * rec + (size_t)round_up_i(l.L, 4) * 4 + (size_t)8 * (NT * (NT + 1) / 2) * 8 +
             (size_t)8 * NT * 4;
    return l;
}

// Largest tile (output pixels, then fewer halo pixels) within the budget and
// at most 40 pixels (5 per warp): larger tiles (6 x 8) measured slower on the
// burst-shaped workload (6.4 against 5.4 ms), 32 pixels the same.
static MmaLayout choose_mma_layout(int NT, const Geom &g, size_t budget) {
    MmaLayout best{};
    for (int TY = 1; TY <= 10; ++TY)
        for (int TX = 1; TX <= 16; ++TX) {
            MmaLayout l = mma_layout(NT, g, TY, TX);
            if (l.smem > budget || TY * TX > 40) continue;
            const long long px = (long long)TY * TX, bpx = (long long)best.TY * best.TX;
            if (px > bpx || (px == bpx && (long long)l.RY * l.RX < (long long)best.RY * best.RX)) best = l;
        }
    return best;
}

template <int NT, bool F16>
static cudaError_t run_cov_mma_plain(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                                     cudaStream_t s) {
    // Two CTAs per SM share its shared memory for NT = 16.
    const size_t budget = NT == 16 ? 110 * 1024 : 220 * 1024;
    const MmaLayout lay = choose_mma_layout(NT, g, budget);
    if (lay.TY == 0) return cudaErrorInvalidConfiguration;
    cudaError_t e =
        cudaFuncSetAttribute(k_cov_mma<NT, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cov_mma<NT, F16>, 256, lay.smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int tilesY = (g.Ho + lay.TY - 1) / lay.TY;
    const long long ntiles = (long long)tilesY * ((g.Wo + lay.TX - 1) / lay.TX);
    if (ntiles == 0) return cudaSuccess;
    const long long grid = std::min<long long>(ntiles, (long long)per_sm * device_sm_count());
    k_cov_mma<NT, F16><<<(unsigned)grid, 256, lay.smem, s>>>(z, n, g, mask, C, lay, ntiles, tilesY);
    return cudaGetLastError();
}

cudaError_t launch_covariance_bf16(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                                   cudaStream_t s) {
    if (n > 32) return cudaErrorInvalidValue;
    if (n <= 16) return run_cov_mma_plain<16, false>(z, n, g, mask, C, s);
    return run_cov_mma_plain<32, false>(z, n, g, mask, C, s);
}

cudaError_t launch_covariance_fp16(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                                   cudaStream_t s) {
    if (n > 32) return cudaErrorInvalidValue;
    if (n <= 16) return run_cov_mma_plain<16, true>(z, n, g, mask, C, s);
    return run_cov_mma_plain<32, true>(z, n, g, mask, C, s);
}

}  // namespace plk
