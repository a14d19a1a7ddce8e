// Phase cosine similarity gamma_s (Sec. III-C, eq. (phase-cosine-sim)): per
// output pixel p, the median over the neighbours x of a disk of radius r of
//   s(p, x) = (1/N_ifg) sum_{(a,b)} cos((phi_b - phi_a)(p) - (phi_b - phi_a)(x)),
// the sum over the nearest-3 network of the M dates (1 <= b - a <= 3).
//
// With unit phasors v = e^{j phi} and w_i = v_i(p) conj(v_i(x)), each term is
// Re(w_b conj(w_a)), so one pass over the dates with w in registers gives the
// three diagonals of the network: per date and neighbour, 4 scalar operations
// for w and 3 packed FP32x2 fused multiply-adds (fma.rn.f32x2) for the terms,
// the centre's phasors held in registers.
//
// A CTA owns a TY x TX tile of output pixels and holds the tile plus an
// r-pixel halo as phasors in shared memory, pixel-major: one record of S
// words per pixel, the phasors of MP dates (MP >= M; dates M.. are zero, so
// they add exactly nothing to any network term and the date loop needs no
// guards), padded to S = 4 x odd words so a record is read in 16-byte loads
// with immediate offsets.  Records are made once per tile with sincosf;
// pixels outside the image or with a non-finite phase get NaN phasors, whose
// similarities are NaN and left out.  A warp owns one output pixel at a
// time: its lanes split the disk's neighbours and keep their similarities in
// registers as order-preserving 32-bit keys.  The neighbour list is dealt
// out by record index mod 8 (eight 16-byte bank groups), so the eight lanes
// of every 16-byte load phase read distinct bank groups; residues that run
// out leave holes.  The median is then selected exactly and warp-uniformly:
// bisection on the key range, each count one warp reduction, stopped as soon
// as one key is left in range (about log2 of the neighbour count steps), and
// the next key for an even count.

#include <algorithm>

#include "f32x2.cuh"
#include "plk_internal.cuh"

namespace plk {

// float -> uint32 with the same order (negative values reversed).
__device__ __forceinline__ uint32_t order_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return b ^ ((b >> 31) ? 0xffffffffu : 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xffffffffu));
}


constexpr int kSimHole = -0x7fffffff;  // an unused slot of the neighbour list

template <int MP, int KT>
__global__ void __launch_bounds__(512) k_phase_sim(const float *__restrict__ phase, int M, int Ho, int Wo, int r,
                                                   int TY, int TX, int S, int nlist, float inv_nifg,
                                                   float *__restrict__ gamma_s) {
    static_assert(MP % 2 == 0, "dates are read in pairs");
    extern __shared__ __align__(16) unsigned char smem[];
    const int HY = TY + 2 * r, HX = TX + 2 * r, HP = HY * HX;
    float *tile = reinterpret_cast<float *>(smem);              // [HP][S]: phasor pairs (cos, sin) per date
    int *off = reinterpret_cast<int *>(tile + (size_t)HP * S);  // [nlist] record offsets (words) or holes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const long long plane = (long long)Ho * Wo;
    const float qnan = __int_as_float(0x7fffffff);
    for (int j = threadIdx.x; j < nlist; j += blockDim.x) off[j] = kSimHole;
    __syncthreads();
    // the disk's offsets (dy, dx), 0 < dy^2 + dx^2 <= r^2: the m-th offset of residue
    // class b = (dy*HX + dx) mod 8 goes to slot 8m + b
    if (threadIdx.x == 0) {
        int fill[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dy * dy + dx * dx <= r * r && (dy || dx)) {
                    const int rec = dy * HX + dx, b = rec & 7;
                    off[8 * fill[b] + b] = rec * S;
                    ++fill[b];
                }
    }
    const int tiles_x = (Wo + TX - 1) / TX;
    const int ntiles = ((Ho + TY - 1) / TY) * tiles_x;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = t / tiles_x, tx = t - (t / tiles_x) * tiles_x;
        const int y0 = ty * TY - r, x0 = tx * TX - r;
        __syncthreads();  // the previous tile's phasors are no longer read (and the offsets are written)
        for (int hp = threadIdx.x; hp < HP; hp += blockDim.x) {
            const int hy = hp / HX, hx = hp - (hp / HX) * HX;
            const int y = y0 + hy, x = x0 + hx;
            const bool in = y >= 0 && y < Ho && x >= 0 && x < Wo;
            const float *src = phase + (in ? (long long)y * Wo + x : 0);
            float4 *rec = reinterpret_cast<float4 *>(tile + (size_t)hp * S);
            float ph[MP];  // every date's load in flight before the first sincosf
#pragma unroll
            for (int i = 0; i < MP; ++i) ph[i] = (in && i < M) ? __ldg(src + i * plane) : qnan;
#pragma unroll
            for (int q = 0; q < MP / 2; ++q) {
                float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;  // dates >= M: zero phasors
                if (2 * q < M) sincosf(ph[2 * q], &s0, &c0);  // non-finite -> NaN
                if (2 * q + 1 < M) sincosf(ph[2 * q + 1], &s1, &c1);
                rec[q] = make_float4(c0, s0, c1, s1);
            }
        }
        __syncthreads();
        for (int px = warp; px < TY * TX; px += nwarp) {
            const int cy = px / TX, cx = px - (px / TX) * TX;
            const int gy = ty * TY + cy, gx = tx * TX + cx;
            if (gy >= Ho || gx >= Wo) continue;  // the same for the whole warp
            const float *ctr = tile + (size_t)((cy + r) * HX + (cx + r)) * S;
            float2 vp[MP];
            bool ok = true;
#pragma unroll
            for (int q = 0; q < MP / 2; ++q) {
                const float4 v2 = reinterpret_cast<const float4 *>(ctr)[q];
                vp[2 * q] = make_float2(v2.x, v2.y);
                vp[2 * q + 1] = make_float2(v2.z, v2.w);
                ok &= !isnan(v2.x) && !isnan(v2.z);  // zero beyond M
            }
            uint32_t key[KT];
            int nv = 0;
            uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
            for (int u = 0; u < KT; ++u) {
                key[u] = 0xffffffffu;  // above every finite key: never counted
                const int j = lane + 32 * u;
                const int o = j < nlist ? off[j] : kSimHole;
                if (o != kSimHole && ok) {
                    const float4 *nb = reinterpret_cast<const float4 *>(ctr + o);
                    unsigned long long w[MP];  // w = v_p conj(v_x), packed (re, im)
#pragma unroll
                    for (int q = 0; q < MP / 2; ++q) {
                        const float4 x2 = nb[q];
                        w[2 * q] = pack2(fmaf(vp[2 * q].x, x2.x, vp[2 * q].y * x2.y),
                                         fmaf(vp[2 * q].y, x2.x, -vp[2 * q].x * x2.y));
                        w[2 * q + 1] = pack2(fmaf(vp[2 * q + 1].x, x2.z, vp[2 * q + 1].y * x2.w),
                                             fmaf(vp[2 * q + 1].y, x2.z, -vp[2 * q + 1].x * x2.w));
                    }
                    // the network terms Re(w_i conj(w_{i-d})) = w_i.re w_j.re + w_i.im w_j.im,
                    // d = 1..3: one packed accumulator per d, halves added at the end
                    unsigned long long a1 = 0ull, a2 = 0ull, a3 = 0ull;  // (0.f, 0.f)
#pragma unroll
                    for (int i = 1; i < MP; ++i) {
                        a1 = fma2(w[i], w[i - 1], a1);
                        if (i >= 2) a2 = fma2(w[i], w[i - 2], a2);
                        if (i >= 3) a3 = fma2(w[i], w[i - 3], a3);
                    }
                    const float acc = hsum2(a1) + hsum2(a2) + hsum2(a3);
                    if (!isnan(acc)) {
                        key[u] = order_key(acc);
                        ++nv;
                        kmin = min(kmin, key[u]);
                        kmax = max(kmax, key[u]);
                    }
                }
            }
            nv = (int)__reduce_add_sync(0xffffffffu, (unsigned)nv);
            float g = qnan;
            if (nv > 0) {  // warp-uniform from here on
                // Invariant: below = #{key < lo} <= k < upto = #{key <= hi}.
                uint32_t lo = __reduce_min_sync(0xffffffffu, kmin), hi = __reduce_max_sync(0xffffffffu, kmax);
                const int k = (nv - 1) / 2;  // lower median
                int below = 0, upto = nv;
                while (upto - below > 1 && lo < hi) {
                    const uint32_t mid = lo + ((hi - lo) >> 1);
                    unsigned c = 0;
#pragma unroll
                    for (int u = 0; u < KT; ++u) c += key[u] <= mid;
                    c = __reduce_add_sync(0xffffffffu, c);
                    if ((int)c > k) {
                        hi = mid;
                        upto = (int)c;
                    } else {
                        lo = mid + 1;
                        below = (int)c;
                    }
                }
                if (lo < hi) {  // one key left in [lo, hi]: the smallest key >= lo
                    uint32_t m = 0xffffffffu;
#pragma unroll
                    for (int u = 0; u < KT; ++u)
                        if (key[u] >= lo) m = min(m, key[u]);
                    lo = __reduce_min_sync(0xffffffffu, m);
                }
                float med = key_value(lo);
                if ((nv & 1) == 0) {  // the mean of the two middle values
                    unsigned c = 0;
                    uint32_t nxt = 0xffffffffu;
#pragma unroll
                    for (int u = 0; u < KT; ++u) {
                        c += key[u] <= lo;
                        if (key[u] > lo) nxt = min(nxt, key[u]);
                    }
                    c = __reduce_add_sync(0xffffffffu, c);
                    nxt = __reduce_min_sync(0xffffffffu, nxt);
                    med = 0.5f * (med + key_value((int)c >= k + 2 ? lo : nxt));
                }
                g = med * inv_nifg;
            }
            if (lane == 0) gamma_s[(long long)gy * Wo + gx] = g;
        }
    }
}

int phase_sim_disk_count(int r) {
    int n = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) n += (dy * dy + dx * dx <= r * r) && (dy || dx);
    return n;
}

// Dates held per record (a compile-time bound >= M).
static int sim_dates(int M) { return M <= 8 ? 8 : M <= 16 ? 16 : M <= 24 ? 24 : 32; }

// Length of the neighbour list dealt out by record index mod 8 (holes included).
static int sim_list_length(int r, int HX) {
    int fill[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx)
            if (dy * dy + dx * dx <= r * r && (dy || dx)) ++fill[(dy * HX + dx) & 7];
    return 8 * *std::max_element(fill, fill + 8);
}

template <int MP>
static cudaError_t launch_sim_mp(const float *phase, int M, int Ho, int Wo, int r, int TY, int TX, int S,
                                 int nlist, size_t smem, float inv_nifg, float *gamma_s, cudaStream_t s) {
    using Kern = void (*)(const float *, int, int, int, int, int, int, int, int, float, float *);
    const int kt = (nlist + 31) / 32;
    Kern kern = kt <= 2 ? k_phase_sim<MP, 2> : kt <= 5 ? k_phase_sim<MP, 5> : kt <= 10 ? k_phase_sim<MP, 10>
                                                                                  : k_phase_sim<MP, 16>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = 512;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long ntiles = (long long)((Ho + TY - 1) / TY) * ((Wo + TX - 1) / TX);
    const long long grid = std::min<long long>(ntiles, (long long)device_sm_count() * per_sm);
    kern<<<(unsigned)grid, threads, smem, s>>>(phase, M, Ho, Wo, r, TY, TX, S, nlist, inv_nifg, gamma_s);
    return cudaGetLastError();
}

cudaError_t launch_phase_similarity(const float *phase, int M, int Ho, int Wo, int r, float *gamma_s,
                                    cudaStream_t s) {
    if ((long long)Ho * Wo == 0) return cudaSuccess;
    const int MP = sim_dates(M);
    // record of a pixel: 2 MP words rounded up to 4 x odd words
    int S = (2 * MP + 3) / 4 * 4;
    if ((S / 4) % 2 == 0) S += 4;
    // Largest tile whose records and neighbour list fit in shared memory.
    static const int shapes[][2] = {{16, 32}, {16, 16}, {8, 16}, {8, 8}, {4, 8}};
    int TY = 0, TX = 0, nlist = 0;
    size_t smem = 0;
    for (const auto &sh : shapes) {
        const int nl = sim_list_length(r, sh[1] + 2 * r);
        const size_t tb = (size_t)S * (sh[0] + 2 * r) * (sh[1] + 2 * r) * sizeof(float) + (size_t)nl * sizeof(int);
        if (tb <= 227 * 1024) {
            TY = sh[0];
            TX = sh[1];
            nlist = nl;
            smem = tb;
            break;
        }
    }
    if (TY == 0 || (nlist + 31) / 32 > 16) return cudaErrorInvalidConfiguration;
    int nifg = 0;
    for (int d = 1; d <= 3; ++d) nifg += std::max(M - d, 0);
    const float inv = 1.0f / (float)nifg;
    switch (MP) {
        case 8: return launch_sim_mp<8>(phase, M, Ho, Wo, r, TY, TX, S, nlist, smem, inv, gamma_s, s);
        case 16: return launch_sim_mp<16>(phase, M, Ho, Wo, r, TY, TX, S, nlist, smem, inv, gamma_s, s);
        case 24: return launch_sim_mp<24>(phase, M, Ho, Wo, r, TY, TX, S, nlist, smem, inv, gamma_s, s);
        default: return launch_sim_mp<32>(phase, M, Ho, Wo, r, TY, TX, S, nlist, smem, inv, gamma_s, s);
    }
}

}  // namespace plk
