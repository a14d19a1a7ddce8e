// S4-S6 kernels over packed coherences: one NP-lane group per pixel (32/NP
// pixels a warp for NP = 8 and 16, one pixel a warp for rows of 20, 24, 28 and
// 32 entries), a single-precision solve, and a double-precision re-solve of the
// pixels it flags (see emi.cuh).
#include "emi.cuh"

namespace plk {

// Row of the coherence cached in shared memory (one slot per lane), gathered
// once from the packed triangle, already padded (identity rows and zero
// columns beyond n), and re-read from there with 16-byte loads.
template <int NP>
struct SmemRow {
    static constexpr bool kPadded = true;
    const cpx<float> *row;  // this lane's NP entries, 16-byte aligned
    __device__ __forceinline__ cpx<float> operator()(int k) const { return row[k]; }
    __device__ __forceinline__ void all(cpx<float> (&c)[NP]) const {
        const uint4 *src = reinterpret_cast<const uint4 *>(row);
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) {
            const uint4 v = src[q];
            memcpy(&c[2 * q], &v, 16);
        }
    }
};

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

// Work area of the double-precision re-solve (kEmiWorkBytes, one per context,
// batch stack or allocation-free call): the single-precision pass appends each
// pixel it flags to the pending list, and the re-solve's warps take list
// entries two groups at a time from a cursor, so the pending pixels spread
// evenly over every resident group whatever their layout, and no warp walks
// the status array.  When more pixels are flagged than the list holds, the
// re-solve falls back to the status scan: warps take 32-pixel chunks of the
// status array in turn, chunk c holding pixels c, c + nchunks, ..., c + 31
// nchunks (pending pixels cluster in space, and interleaving spreads a cluster
// over many chunks and warps).  k_reset_counter zeroes the three counters
// before the single-precision pass (stream order).
__global__ void k_reset_counter(unsigned long long *c) {
    if (threadIdx.x < 3) c[threadIdx.x] = 0;
}

__device__ __forceinline__ long long next_chunk(unsigned long long *counter, int lane, unsigned long long inc = 1) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(counter, inc);
    return (long long)__shfl_sync(0xffffffffu, c, 0);
}

// Append pixel p to the pending list (one lane of its group).
__device__ __forceinline__ void append_pending(unsigned long long *work, long long p) {
    const unsigned long long i = atomicAdd(work + 1, 1ull);
    if (i < (unsigned long long)kPendCap) pending_list(work)[i] = (unsigned)p;
}

// The re-solve's loop over pending pixels: solve(p) for each, one NP-lane
// group at a time; list mode when the list held every flagged pixel, the
// status scan otherwise.
template <int NP, class Solve>
__device__ __forceinline__ void for_each_pending(unsigned long long *work, bool use_list, long long npx,
                                                 const uint8_t *status, int lane, const Solve &solve) {
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    constexpr int G = kPow2 ? 32 / NP : 1;  // rows of 20, 24 or 28 entries: one pixel a warp
    const int grp = kPow2 ? lane / NP : 0;
    const unsigned long long cnt = use_list ? *(volatile unsigned long long *)(work + 1) : ~0ull;
    if (cnt <= (unsigned long long)kPendCap) {
        const unsigned *lst = pending_list(work);
        for (;;) {
            const long long b0 = next_chunk(work + 2, lane, (unsigned long long)G);
            if (b0 >= (long long)cnt) break;
            const long long i = b0 + grp;
            if (i < (long long)cnt) solve((long long)lst[i]);
            __syncwarp();
        }
        return;
    }
    const long long nchunks = (npx + 31) / 32;
    for (;;) {
        const long long base = next_chunk(work, lane);
        if (base >= nchunks) break;
        const long long pl = base + (long long)lane * nchunks;  // interleaved: clusters spread over chunks
        const bool pend = pl < npx && status[pl] == (uint8_t)kPending;
        unsigned bal = __ballot_sync(0xffffffffu, pend);
        while (bal) {
            int mine = -1;
#pragma unroll
            for (int gg = 0; gg < G; ++gg) {
                if (bal) {
                    const int b = __ffs(bal) - 1;
                    if (gg == grp) mine = b;
                    bal &= bal - 1u;
                }
            }
            if (mine >= 0) solve(base + (long long)mine * nchunks);
            __syncwarp();
        }
    }
}

// Single-precision pass: one NP-lane group per pixel.  Pixels the solve flags
// get status kPending and no other output.
// Rows of 20, 24 and 28 entries (emi_row_length) run one pixel a warp with the
// lanes past the row idle: a solve costs about n times the row length, so they
// save the padded work of 32-entry rows for 17 <= N <= 28.
// Warps per CTA of the single-precision pass: 2 for rows beyond 16 entries,
// whose per-lane shared memory would otherwise pass the 48 KB a CTA may
// declare statically.  CTAs per SM the kernel is register-budgeted for: 16
// warps an SM at 128 registers for rows of up to 24 entries (4 CTAs of 4 warps,
// 8 of 2), 12 warps for 28 and 32 (6 CTAs of 2, up to 168 registers: at 128
// they spill and run 4% slower at N = 28, while 16 warps gain 12% at N = 20).
template <int NP>
struct EmiWarps {
    static constexpr int value = NP > 16 ? 2 : 4;
};
template <int NP>
struct EmiMinBlocks {
    static constexpr int value = NP > 24 ? 6 : (NP > 16 ? 8 : 4);
};

// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (the
// source is then not read but must be a valid pointer).
__device__ __forceinline__ void cp_async8_emi(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Prefetch of the packed coherences: the warp copies the triangles of its
// next G pixels (G * N(N+1)/2 entries, one contiguous run) into shared memory
// while it solves the current ones, so the gather of a pixel's rows reads
// shared memory instead of waiting on global loads (two slots a warp; with the
// two-warp CTAs of rows beyond 16 entries they fit the static budget up to 32).
template <int NP>
struct EmiPrefetch {
    static constexpr int G = ((NP & (NP - 1)) == 0) ? 32 / NP : 1;
    static constexpr int elems = G * NP * (NP + 1) / 2;
};

template <int NP>
__global__ void __launch_bounds__(EmiWarps<NP>::value * 32, EmiMinBlocks<NP>::value) k_emi32(const float2 *__restrict__ C, int n, long long npx,
                                                          int ref, const EmiParams prm,
                                                          float *__restrict__ phase, float *__restrict__ tcoh,
                                                          float *__restrict__ lam, uint8_t *__restrict__ status,
                                                          bool use_list) {
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    constexpr int kW = EmiWarps<NP>::value;
    constexpr int G = kPow2 ? 32 / NP : 1;
    // Complex entries per cached row: NP + 2 (16-byte aligned rows whose
    // 16-byte chunks fall in different banks for 8 consecutive lanes).
    constexpr int kRowPitch = NP + 2;
    __shared__ __align__(16) cpx<float> sbuf[kW][32];
    __shared__ __align__(16) cpx<float> rowcache[kW * 32 * kRowPitch];
    __shared__ __align__(16) float2 pf[kW][2][EmiPrefetch<NP>::elems];
    // Rows of G^{-1}, one per lane; the pitch NP + 4 puts the 16-byte chunks of
    // 8 consecutive lanes in different banks.
    constexpr int kGPitch = NP + 4;
    __shared__ __align__(16) float gsm[kW * 32 * kGPitch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = kPow2 ? lane / NP : 0, r = lane - grp * NP;
    const int glane0 = grp * NP;
    const unsigned gmask = (!kPow2 || NP == 32) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    const long long step = (long long)gridDim.x * kW * G;
    cpx<float> *myrow = rowcache + (size_t)(warp * 32 + lane) * kRowPitch;

    // Copy the packed triangles of pixels b .. b + G - 1 (those below npx)
    // into prefetch slot `slot`; one commit group per call, empty past the end.
    auto prefetch = [&](long long b, int slot) {
        const long long cnt = b < npx ? ((npx - b < G) ? (npx - b) : G) * nt : 0;
        const float2 *src = C + (b < npx ? b : 0) * nt;
        for (int e = lane; e < G * nt; e += 32) {
            const bool ok = e < cnt;
            cp_async8_emi(&pf[warp][slot][e], ok ? src + e : C, ok ? 8 : 0);
        }
        cp_async_commit();
    };
    long long base = ((long long)blockIdx.x * kW + warp) * G;
    int slot = 0;
    prefetch(base, 0);
    for (; base < npx; base += step, slot ^= 1) {
        const long long p = base + grp;
        const bool valid = p < npx;
        prefetch(base + step, slot ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this iteration's copies have landed
        __syncwarp();
        const float2 *Cpix = &pf[warp][slot][grp * nt];
        bool nan = false;
        if (valid && r < n) nan = isnan(Cpix[packed_index(n, r, r)].x);
        nan = __any_sync(gmask, nan);
        if (valid && !nan) {
            // Gather row r once: entries k >= r are contiguous in the packed
            // triangle, entries k < r are the conjugates down column r.
            {
                // The lanes of a group differ in which side of the diagonal
                // an entry lies, so the gather picks the packed index and the
                // sign without branching.  Rows of 8 and 16 entries gather into
                // registers and store 16 bytes at a time; wider rows store
                // each entry from a loop that is not unrolled (short code:
                // 6% faster at N = 20 and 28, where the kernel is sensitive to
                // its instruction footprint).
                const int base_r = r * n - r * (r - 1) / 2 - r;  // + k for k >= r
                int idx_col = r;                                  // packed index of (k, r), k = 0
                auto entry = [&](int k) {
                    const bool up = k >= r, in = r < n && k < n;
                    const float2 c = Cpix[in ? (up ? base_r + k : idx_col) : 0];
                    idx_col += (in && !up) ? n - k - 1 : 0;
                    return in ? mk<float>(c.x, up ? c.y : -c.y) : mk<float>((k == r) ? 1.f : 0.f, 0.f);
                };
                if constexpr (NP > 16) {
#pragma unroll 1
                    for (int k = 0; k < NP; ++k) myrow[k] = entry(k);
                } else {
                    cpx<float> v[NP];
#pragma unroll
                    for (int k = 0; k < NP; ++k) v[k] = entry(k);
                    uint4 *dst = reinterpret_cast<uint4 *>(myrow);
#pragma unroll
                    for (int q = 0; q < NP / 2; ++q) {
                        uint4 w;
                        memcpy(&w, &v[2 * q], 16);
                        dst[q] = w;
                    }
                }
            }
            SmemRow<NP> ld{myrow};
            const PixelResult res = emi_solve<NP, float, SmemRow<NP>, true>(
                ld, r, n, ref, prm, &sbuf[warp][glane0], gmask, glane0, false, gsm + (warp * 32 + lane) * kGPitch);
            if (res.flag) {
                if (r == 0) {
                    status[p] = (uint8_t)kPending;
                    if (use_list) append_pending(prm.work, p);
                }
            } else {
                if (r < n) phase[(long long)r * npx + p] = res.phase;
                if (r == 0) {
                    if (tcoh) tcoh[p] = res.tcoh;
                    if (lam) lam[p] = res.lam;
                    status[p] = (uint8_t)res.status;
                }
            }
        } else if (valid) {
            if (r < n) phase[(long long)r * npx + p] = __int_as_float(0x7fc00000);
            if (r == 0) {
                if (tcoh) tcoh[p] = __int_as_float(0x7fc00000);
                if (lam) lam[p] = __int_as_float(0x7fc00000);
                status[p] = PLK_PX_NODATA;
            }
        }
        __syncwarp();  // the slot is free for the copies issued next iteration
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Double-precision re-solve of the pixels left pending, one per NP-lane group
// as for_each_pending hands them out.
template <int NP>
__global__ void __launch_bounds__(kEmiWarps * 32) k_emi64(const float2 *__restrict__ C, int n, long long npx,
                                                          int ref, const EmiParams prm,
                                                          float *__restrict__ phase, float *__restrict__ tcoh,
                                                          float *__restrict__ lam, uint8_t *__restrict__ status,
                                                          bool use_list) {
    __shared__ __align__(16) cpx<double> sbuf[kEmiWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    const int grp = kPow2 ? lane / NP : 0, r = lane - grp * NP;
    const int glane0 = grp * NP;
    const unsigned gmask = (!kPow2 || NP == 32) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    for_each_pending<NP>(prm.work, use_list, npx, status, lane, [&](long long p) {
        PackedRow<double> ld{C + p * nt, n, r};
        const PixelResult res = emi_solve_mixed<NP>(ld, r, n, ref, prm, &sbuf[warp][glane0], gmask, glane0);
        if (r < n) phase[(long long)r * npx + p] = res.phase;
        if (r == 0) {
            if (tcoh) tcoh[p] = res.tcoh;
            if (lam) lam[p] = res.lam;
            status[p] = (uint8_t)res.status;
        }
    });
}

// Row source held in registers (indexed with compile-time k after inlining).
template <int NP, class T>
struct RegRow {
    cpx<T> c[NP];
    __device__ __forceinline__ cpx<T> operator()(int k) const { return c[k]; }
};

// Double-precision row source in shared memory (one slot per lane): the
// re-solve reads it to form A and again for the start vector and gamma_t, so
// it holds no registers in between.
template <int NP>
struct SmemRowD {
    const cpx<double> *row;
    __device__ __forceinline__ cpx<double> operator()(int k) const { return row[k]; }
};

// Warps per CTA of the stack re-solve: 2 for rows beyond 16 entries, whose
// per-lane row slots would otherwise pass the 48 KB a CTA may declare statically.
template <int NP>
struct Emi64Warps {
    static constexpr int value = NP > 16 ? 2 : 4;
};

// Sum of exact products in a pair of floats (hi + lo): the product a*b is
// split exactly into p + e (p = fl(a*b), e = fma(a, b, -p)), and p is added to
// hi by Knuth's TwoSum, its rounding error going to lo with e.  The
// intrinsics keep the compiler from contracting or reordering any step.  Over
// the few dozen looks of a window the pair carries about 46 significant bits,
// as a double-precision sum of the same products does (each product of two
// single-precision samples is exact in double precision); GB300's FP32 pipes
// do this several times faster than its FP64 units do the double sum.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ void f2_add_prod(F2 &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double f2_value(const F2 &a) { return (double)a.hi + (double)a.lo; }

// Double-precision re-solve for the mini-stack path: the coherence row of a
// pending pixel is recomputed from the SLC stack over its SHP neighbourhood
// with exact products and float-pair sums (F2), carried to double precision,
// so the solve sees the coherence an FP64 reference computes instead of the
// single-precision one.
template <int NP>
__global__ void __launch_bounds__(Emi64Warps<NP>::value * 32) k_emi64_stack(const __grid_constant__ Planes z, const Geom g,
                                                                const uint64_t *__restrict__ mask, int n,
                                                                long long npx, int ref, const EmiParams prm,
                                                                float *__restrict__ phase, float *__restrict__ tcoh,
                                                                float *__restrict__ lam,
                                                                uint8_t *__restrict__ status, bool use_list) {
    constexpr int E = 16 / sizeof(cpx<double>);
    constexpr int kW = Emi64Warps<NP>::value;
    // Row slots with a pitch of NP + 1 entries: the 16-byte entries of 8
    // consecutive lanes fall in different banks.
    constexpr int kPitch = NP + 1;
    __shared__ __align__(16) cpx<double> sbuf[kW][32];
    __shared__ __align__(16) cpx<double> rows[kW * 32 * kPitch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    const int grp = kPow2 ? lane / NP : 0, r = lane - grp * NP;
    const int glane0 = grp * NP;
    const unsigned gmask = (!kPow2 || NP == 32) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    for_each_pending<NP>(prm.work, use_list, npx, status, lane, [&](long long p) {
        const int oy = (int)(p / g.Wo), ox = (int)(p - (p / g.Wo) * g.Wo);
        const int cy = oy * g.sy + g.sy / 2, cx = ox * g.sx + g.sx / 2;
        const uint64_t *mw = mask + p * g.nwords;
        F2 re[NP], im[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) re[k] = im[k] = F2{0.f, 0.f};
        int b = 0;
        uint64_t word = __ldg(mw);
        for (int dy = -g.hy; dy <= g.hy; ++dy)
            for (int dx = -g.hx; dx <= g.hx; ++dx, ++b) {
                if ((b & 63) == 0 && b > 0) word = __ldg(mw + (b >> 6));
                if (!((word >> (b & 63)) & 1ull)) continue;
                const long long q = (long long)(cy + dy) * g.W + (cx + dx);
                float2 zr = make_float2(0.f, 0.f);
                if (r < n) zr = __ldg(z.p[r] + q);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    if (k < n) {
                        const float2 zk = __ldg(z.p[k] + q);
                        // z_r conj(z_k) = (xr xk + yr yk) + j (yr xk - xr yk)
                        f2_add_prod(re[k], zr.x, zk.x);
                        f2_add_prod(re[k], zr.y, zk.y);
                        f2_add_prod(im[k], zr.y, zk.x);
                        f2_add_prod(im[k], -zr.x, zk.y);
                    }
                }
            }
        // The sums in double precision go straight to this lane's row slot,
        // then are normalised there: C_rk = S_rk s_r s_k with s_i =
        // 1/sqrt(S_ii) (0 when S_ii = 0), C_rr = 1; one square root per lane.
        cpx<double> *slot = rows + (warp * 32 + lane) * kPitch;
        double d_own = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            slot[k] = mk<double>(f2_value(re[k]), f2_value(im[k]));
            if (k == r) d_own = f2_value(re[k]);
        }
        cpx<double> *buf = &sbuf[warp][glane0];
        const double s_own = (d_own > 0.0) ? 1.0 / sqrt(d_own) : 0.0;
        buf[r] = mk<double>(s_own, 0.0);
        __syncwarp(gmask);
        const uint4 *src = reinterpret_cast<const uint4 *>(buf);
#pragma unroll
        for (int q4 = 0; q4 < NP / E; ++q4) {
            const uint4 v = src[q4];
            cpx<double> sk[E];
            memcpy(sk, &v, 16);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = q4 * E + e;
                const double sc = s_own * sk[e].x;
                const cpx<double> c = slot[k];
                slot[k] = (k == r) ? mk<double>(1.0, 0.0) : mk<double>(c.x * sc, c.y * sc);
            }
        }
        __syncwarp(gmask);
        const PixelResult res = emi_solve_mixed<NP>(SmemRowD<NP>{slot}, r, n, ref, prm, buf, gmask, glane0);
        if (r < n) phase[(long long)r * npx + p] = res.phase;
        if (r == 0) {
            if (tcoh) tcoh[p] = res.tcoh;
            if (lam) lam[p] = res.lam;
            status[p] = (uint8_t)res.status;
        }
    });
}

template <int NP>
static cudaError_t run_emi(const float2 *C, int n, long long npx, int ref, const EmiParams &prm, float *phase,
                           float *tcoh, float *lam, uint8_t *status, cudaStream_t s, Prof *prof,
                           const StackSource *src) {
    constexpr int G = (NP & (NP - 1)) ? 1 : 32 / NP;
    constexpr int NP64 = NP;
    constexpr int W = EmiWarps<NP>::value;
    const long long cap = (long long)device_sm_count() * 64 / W;
    long long blocks = ((npx + G - 1) / G + W - 1) / W;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    // pixel indices of the pending list are 32-bit
    const bool use_list = npx <= 0xffffffffLL;
    if (prm.fp64_resolve) k_reset_counter<<<1, 32, 0, s>>>(prm.work);
    if (prof) prof->begin("phase_link_fp32", s);
    k_emi32<NP><<<(unsigned)blocks, W * 32, 0, s>>>(C, n, npx, ref, prm, phase, tcoh, lam, status,
                                                           use_list && prm.fp64_resolve);
    cudaError_t e = cudaGetLastError();
    if (prof) prof->end(s);
    if (e != cudaSuccess || !prm.fp64_resolve) return e;
    // CTAs of w warps, no more than are resident at the re-solve's register
    // use (255 a thread: 8 warps an SM)
    auto grid64 = [&](int w) {
        const long long b = ((npx + 31) / 32 + w - 1) / w, cap = (long long)device_sm_count() * (8 / w);
        return (unsigned)(b > cap ? cap : (b < 1 ? 1 : b));
    };
    constexpr int W64 = Emi64Warps<NP64>::value;
    if (prof) prof->begin("phase_link_fp64", s);
    if (src)
        k_emi64_stack<NP64><<<grid64(W64), W64 * 32, 0, s>>>(*src->z, *src->g, src->mask, n, npx, ref,
                                                                          prm, phase, tcoh, lam, status, use_list);
    else
        k_emi64<NP64><<<grid64(kEmiWarps), kEmiWarps * 32, 0, s>>>(C, n, npx, ref, prm, phase, tcoh, lam, status,
                                                                    use_list);
    e = cudaGetLastError();
    if (prof) prof->end(s);
    return e;
}

cudaError_t launch_phase_link(const float2 *C, int n, long long npx, int ref, const EmiParams &prm,
                              float *phase, float *tcoh, float *lam, uint8_t *status, cudaStream_t s, Prof *prof,
                              const StackSource *src, const Schedule *sch) {
    if (npx == 0) return cudaSuccess;
    // Lanes per pixel: the smallest group that holds a row, unless the
    // schedule asks for a wider one (fewer pixels per warp).
    int np = emi_row_length(n);
    if (sch && sch->emi_np >= np && emi_row_length(sch->emi_np) == sch->emi_np) np = sch->emi_np;
    switch (np) {
        case 8: return run_emi<8>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
        case 16: return run_emi<16>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
        case 20: return run_emi<20>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
        case 24: return run_emi<24>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
        case 28: return run_emi<28>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
        default: return run_emi<32>(C, n, npx, ref, prm, phase, tcoh, lam, status, s, prof, src);
    }
}

}  // namespace plk
