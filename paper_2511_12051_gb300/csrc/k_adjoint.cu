// Adjoint of S3-S5 (coherence -> EMI eigenvector -> referenced phase) with
// the SHP masks frozen: for L = sum_{p,i} w_{p,i} phihat_{p,i}, the gradient
// g(q) with dL = Re sum conj(g) dz over the SLC stack (the convention under
// which g = dL/dRe z + j dL/dIm z).  The coherence is recomputed here, not
// stored by the forward pass.
//
// Per output pixel p (an NP-lane group, lane r owning row r):
//   phihat_i = arg(v_i conj(v_ref)):  g_v,i = w_i j v_i / |v_i|^2 (i != ref),
//     g_v,ref = -(sum_{i != ref} w_i) j v_ref / |v_ref|^2; the common-phase
//     direction j v carries no gradient (the phases are gauge invariant).
//   v = unit eigenvector of A for the simple eigenvalue lambda (A = G^-1 o C,
//     or C itself on the EVD fallback):  dv = -(A - lambda I)^+ dA v, so with
//     u = (A - lambda I + c v v^H)^-1 (g_v - v v^H g_v)  (u orthogonal to v),
//     the gradient on A is GA = -u v^H.
//   A = G^-1 o C:  GC += G^-1 o GA;  R = Re(conj(GA) o C);  GG = -G^-1 R G^-1;
//     G = (1-beta)|C| + beta I:  GC += (1-beta) GG o C/|C|  (off the diagonal,
//     which is constant).
//   C_ik = S_ik / sqrt(S_ii S_kk):  GS_ik = GC_ik / sqrt(S_ii S_kk) (i != k),
//     GS_ii = -(sum_k P_ik + sum_k P_ki) / (2 S_ii), P = Re(conj(GC) o C).
//   H_p = GS + GS^H  (Hermitian, stored as the packed upper triangle).
// Per input pixel q and date i (gather):  g_i(q) = sum over the output
//   pixels p whose window holds q with the mask bit set of (H_p z(q))_i.
#include <algorithm>

#include "emi.cuh"

namespace plk {

namespace {

constexpr int kAdjWarps = 2;

// Row of the coherence cached in shared memory, padded (see k_emi.cu).
template <int NP>
struct AdjRow {
    static constexpr bool kPadded = true;
    const cpx<float> *row;
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

// Publish every lane's row of an NP x NP matrix to the group's buffer.
template <int NP, class S>
__device__ __forceinline__ void publish(const S (&row)[NP], S *mat, int r, unsigned gmask) {
    __syncwarp(gmask);
#pragma unroll
    for (int k = 0; k < NP; ++k) mat[r * NP + k] = row[k];
    __syncwarp(gmask);
}

}  // namespace

// Diagonal sums S_ii = sum over the mask of |z_i(q)|^2, one thread per
// (output pixel, date).
__global__ void __launch_bounds__(256) k_adj_sdiag(const __grid_constant__ Planes z, int n, const Geom g,
                                                   const uint64_t *__restrict__ mask, float *__restrict__ Sd) {
    const long long nout = (long long)g.Ho * g.Wo;
    const long long total = nout * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / nout);
        const long long o = t - (long long)i * nout;
        const int oy = (int)(o / g.Wo), ox = (int)(o - (long long)oy * g.Wo);
        const int cy = oy * g.sy + g.sy / 2, cx = ox * g.sx + g.sx / 2;
        const uint64_t *mw = mask + o * g.nwords;
        float s = 0.f;
        int b = 0;
        for (int dy = -g.hy; dy <= g.hy; ++dy)
            for (int dx = -g.hx; dx <= g.hx; ++dx, ++b) {
                if (!((__ldg(mw + (b >> 6)) >> (b & 63)) & 1ull)) continue;
                const float2 v = __ldg(z.p[i] + (long long)(cy + dy) * g.W + (cx + dx));
                s += v.x * v.x + v.y * v.y;
            }
        Sd[o * n + i] = s;
    }
}

// Per-pixel state of the uncertainty kernel that does not depend on the date:
// in registers, this lane's eigenvector entry and its row of the inverted
// deflated matrix (A - lambda I + c v v^H)^-1; in the group's shared memory
// (UncShared), the coherence row (the lane's row cache), every lane's v, every
// 1/sqrt(S_kk) and G^-1.  Keeping the group-uniform vectors and the rows that
// are only read out of the register file leaves the per-date products room.
template <int NP>
struct AdjPixelState {
    cpx<float> v, mrow[NP];
    float sr, rsr;
    bool evd, live;
};

// Group views of the shared buffers: row r of C (myrow, padded), v and
// 1/sqrt(S_kk) of every lane, G^-1 [NP][NP].
template <int NP>
struct UncShared {
    const cpx<float> *myrow;
    cpx<float> *vg;
    float *rsg;
    float *ginv;
};

template <int NP>
__device__ __forceinline__ void adj_prepare(AdjPixelState<NP> &S, const UncShared<NP> &sh, const float *__restrict__ Sd,
                                            long long p, int r, int n, int ref, const EmiParams &q,
                                            cpx<float> *cbuf, unsigned gmask, int glane0) {
    float *rbuf = reinterpret_cast<float *>(cbuf);
    const AdjRow<NP> ld{sh.myrow};
    S.live = r < n;
    const PixelResult res = emi_solve<NP, float>(ld, r, n, ref, q, cbuf, gmask, glane0, false);
    S.evd = res.evd;
    S.v = S.live ? res.v : mk<float>(0.f, 0.f);
    // G^-1 row, published to the group's matrix.
    {
        float gi[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float m = mag_t(norm2(sh.myrow[k]));
            if (q.beta != 0.f) m = (1.f - q.beta) * m + ((k == r) ? q.beta : 0.f);
            gi[k] = m;
        }
        if (!S.evd) gj_invert<NP, float, float, true>(gi, rbuf, r, n, gmask, 0.f);
        publish<NP, float>(gi, sh.ginv, r, gmask);
    }
    // A row (C, or G^-1 o C) into mrow; lambda = v^H A v.
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const cpx<float> c = sh.myrow[k];
        const float gk = sh.ginv[r * NP + k];
        S.mrow[k] = S.evd ? c : mk<float>(gk * c.x, gk * c.y);
    }
    const cpx<float> av = group_matvec<NP, float>(S.mrow, S.v, cbuf, r, gmask);
    const float lam = group_sum<NP, float>(S.live ? (S.v.x * av.x + S.v.y * av.y) : 0.f, gmask);
    sh.vg[r] = S.v;
    __syncwarp(gmask);
    // (A - lambda I + c v v^H)^-1  (c keeps the deflated matrix well scaled)
    const float cdef = fmaxf(1.f, fabsf(lam));
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        S.mrow[k] = S.mrow[k] + cdef * (S.v * conj(sh.vg[k]));
        if (k == r && S.live) S.mrow[k].x -= lam;
    }
    gj_invert<NP, float, cpx<float>, false>(S.mrow, cbuf, r, n, gmask, 0.f);
    S.sr = S.live ? __ldg(Sd + p * n + r) : 0.f;
    S.rsr = S.sr > 0.f ? rsqrtf(S.sr) : 0.f;
    sh.rsg[r] = S.rsr;
    __syncwarp(gmask);
}

// Row r of H = GS + GS^H for the phase weight wr of this lane's date (the
// weight of the reference date is unused: its phase is 0).  Products over the
// date index stop at n (rows and columns past n are zero).
template <int NP>
__device__ __forceinline__ void adj_h_row(const AdjPixelState<NP> &S, const UncShared<NP> &sh, float wr, int r, int n,
                                          int ref, float beta, cpx<float> *cbuf, cpx<float> *cmat, unsigned gmask,
                                          cpx<float> (&h)[NP]) {
    float *fmat = reinterpret_cast<float *>(cmat);
    // Gradient on v (gauge-free), projected orthogonal to v.
    const float wsum = group_sum<NP, float>(S.live && r != ref ? wr : 0.f, gmask);
    const float m2 = norm2(S.v);
    const float coef = (r == ref) ? -wsum : wr;
    cpx<float> gv = (S.live && m2 > 0.f) ? (coef / m2) * mk<float>(-S.v.y, S.v.x) : mk<float>(0.f, 0.f);
    {
        const cpx<float> t = conj(S.v) * gv;
        const float sx = group_sum<NP, float>(t.x, gmask), sy = group_sum<NP, float>(t.y, gmask);
        gv = gv - S.v * mk<float>(sx, sy);
    }
    // u = (A - lambda I + c v v^H)^-1 g_v  (u orthogonal to v)
    const cpx<float> u = group_matvec<NP, float>(S.mrow, gv, cbuf, r, gmask);

    // GA = -u v^H (row r), then GC (off the diagonal); h holds GC.
#pragma unroll
    for (int k = 0; k < NP; ++k) h[k] = mk<float>(0.f, 0.f) - u * conj(sh.vg[k]);
    if (!S.evd) {
        float T[NP];
        {
            float R[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const cpx<float> c = sh.myrow[k];
                R[k] = h[k].x * c.x + h[k].y * c.y;  // Re(conj(GA) C)
            }
            publish<NP, float>(R, fmat, r, gmask);
        }
        // T = G^-1 R (row r)
#pragma unroll
        for (int k = 0; k < NP; ++k) T[k] = 0.f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (j >= n) break;
            const float gj = sh.ginv[r * NP + j];
#pragma unroll
            for (int k = 0; k < NP; ++k) T[k] += gj * fmat[j * NP + k];
        }
        // GG = -T G^-1 (row r)
        float GG[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) GG[k] = 0.f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (j >= n) break;
#pragma unroll
            for (int k = 0; k < NP; ++k) GG[k] -= T[j] * sh.ginv[j * NP + k];
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const cpx<float> c = sh.myrow[k];
            const float cm2 = norm2(c);
            const cpx<float> ph = cm2 > 0.f ? rsqrtf(cm2) * c : mk<float>(0.f, 0.f);
            h[k] = sh.ginv[r * NP + k] * h[k] + ((1.f - beta) * GG[k]) * ph;
        }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k)
        if (k == r || k >= n || !S.live) h[k] = mk<float>(0.f, 0.f);

    // C -> S.
    {
        float P[NP];
        float rowsum = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const cpx<float> c = sh.myrow[k];
            P[k] = h[k].x * c.x + h[k].y * c.y;
            rowsum += P[k];
        }
        publish<NP, float>(P, fmat, r, gmask);
        float colsum = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) colsum += fmat[i * NP + r];
#pragma unroll
        for (int k = 0; k < NP; ++k) h[k] = (S.rsr * sh.rsg[k]) * h[k];
        if (S.live && S.sr > 0.f) h[r] = mk<float>(-(rowsum + colsum) / (2.f * S.sr), 0.f);
    }

    // H = GS + GS^H (row r)
    publish<NP, cpx<float>>(h, cmat, r, gmask);
#pragma unroll
    for (int k = 0; k < NP; ++k) h[k] = h[k] + conj(cmat[k * NP + r]);
    __syncwarp(gmask);
}

// Coherence row r of pixel p, unit diagonal, into the lane's row cache.
template <int NP>
__device__ __forceinline__ void adj_load_row(cpx<float> *myrow, const float2 *__restrict__ Cpix, int r, int n) {
    const bool live = r < n;
    const int base_r = r * n - r * (r - 1) / 2 - r;
    int idx_col = r;
    cpx<float> v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        v[k] = mk<float>((!live && k == r) ? 1.f : 0.f, 0.f);
        if (live && k < n) {
            if (k >= r) {
                const float2 c = __ldg(Cpix + base_r + k);
                v[k] = mk<float>(c.x, c.y);
            } else {
                const float2 c = __ldg(Cpix + idx_col);
                v[k] = mk<float>(c.x, -c.y);
                idx_col += n - k - 1;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) myrow[k] = v[k];
}

// Per output pixel: H_p from the coherence C (packed), the diagonal sums and
// the phase weights w [n][npx].  Pixels without data get H_p = 0.
template <int NP>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adj_pixel(const float2 *__restrict__ C,
                                                              const float *__restrict__ Sd, int n, long long npx,
                                                              int ref, const EmiParams prm,
                                                              const float *__restrict__ w,
                                                              float2 *__restrict__ Hout) {
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    constexpr int G = kPow2 ? 32 / NP : 1;
    constexpr int kRowPitch = NP + 2;
    constexpr int kGrpBuf = 2 * NP + 2;
    __shared__ __align__(16) cpx<float> sbuf[kAdjWarps][G * kGrpBuf];
    __shared__ __align__(16) cpx<float> rowcache[kAdjWarps * 32 * kRowPitch];
    __shared__ __align__(16) cpx<float> mats[kAdjWarps][32 * NP];  // one NP x NP matrix per group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = kPow2 ? lane / NP : 0, r = lane - grp * NP;  // 24-entry rows: one pixel a warp
    const int glane0 = grp * NP;
    const unsigned gmask = (NP >= 24) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    const long long step = (long long)gridDim.x * kAdjWarps * G;
    cpx<float> *myrow = rowcache + (size_t)(warp * 32 + lane) * kRowPitch;
    cpx<float> *cbuf = &sbuf[warp][grp * kGrpBuf];
    float *rbuf = reinterpret_cast<float *>(cbuf);
    cpx<float> *cmat = &mats[warp][grp * NP * NP];
    float *fmat = reinterpret_cast<float *>(cmat);
    EmiParams q = prm;
    q.fp64_resolve = 0;  // the adjoint differentiates the single-precision solve

    for (long long base = ((long long)blockIdx.x * kAdjWarps + warp) * G; base < npx; base += step) {
        const long long p = base + grp;
        const bool valid = p < npx;
        const float2 *Cpix = C + (valid ? p : 0) * nt;
        const bool live = r < n;
        bool nan = false;
        if (valid && live) nan = isnan(__ldg(Cpix + packed_index(n, r, r)).x);
        nan = __any_sync(gmask, nan);
        if (!valid) continue;
        if (nan) {
            if (live)
                for (int k = r; k < n; ++k) Hout[p * nt + packed_index(n, r, k)] = make_float2(0.f, 0.f);
            continue;
        }
        {
            const int base_r = r * n - r * (r - 1) / 2 - r;
            int idx_col = r;
            cpx<float> v[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                v[k] = mk<float>((!live && k == r) ? 1.f : 0.f, 0.f);
                if (live && k < n) {
                    if (k >= r) {
                        const float2 c = __ldg(Cpix + base_r + k);
                        v[k] = mk<float>(c.x, c.y);
                    } else {
                        const float2 c = __ldg(Cpix + idx_col);
                        v[k] = mk<float>(c.x, -c.y);
                        idx_col += n - k - 1;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) myrow[k] = v[k];
        }
        __syncwarp(gmask);
        const AdjRow<NP> ld{myrow};
        const PixelResult res = emi_solve<NP, float>(ld, r, n, ref, q, cbuf, gmask, glane0, false);
        const cpx<float> v = live ? res.v : mk<float>(0.f, 0.f);

        // Gradient on v (gauge-free), projected orthogonal to v.
        const float wr = live ? __ldg(w + (long long)r * npx + p) : 0.f;
        const float wsum = group_sum<NP, float>(live && r != ref ? wr : 0.f, gmask);
        const float m2 = norm2(v);
        const float coef = (r == ref) ? -wsum : wr;
        cpx<float> gv = (live && m2 > 0.f) ? (coef / m2) * mk<float>(-v.y, v.x) : mk<float>(0.f, 0.f);
        {
            const cpx<float> t = conj(v) * gv;
            const float sx = group_sum<NP, float>(t.x, gmask), sy = group_sum<NP, float>(t.y, gmask);
            gv = gv - v * mk<float>(sx, sy);
        }

        // A row (C, or G^-1 o C) and G^-1 row.
        cpx<float> crow[NP], a[NP];
        float gi[NP];
        load_crow<NP, float>(crow, ld, r, n);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float m = mag_t(norm2(crow[k]));
            if (q.beta != 0.f) m = (1.f - q.beta) * m + ((k == r) ? q.beta : 0.f);
            gi[k] = m;
        }
        if (!res.evd) gj_invert<NP, float, float, true>(gi, rbuf, r, n, gmask, 0.f);
#pragma unroll
        for (int k = 0; k < NP; ++k) a[k] = res.evd ? crow[k] : mk<float>(gi[k] * crow[k].x, gi[k] * crow[k].y);
        // lambda = v^H A v (the eigenvalue the perturbation is about)
        const cpx<float> av = group_matvec<NP, float>(a, v, cbuf, r, gmask);
        const float lam = group_sum<NP, float>(live ? (v.x * av.x + v.y * av.y) : 0.f, gmask);
        // every lane's v
        cpx<float> vv[NP];
        cbuf[r] = v;
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < NP; ++k) vv[k] = cbuf[k];
        __syncwarp(gmask);
        // u = (A - lambda I + c v v^H)^-1 g_v  (c keeps the deflated matrix well scaled)
        const float cdef = fmaxf(1.f, fabsf(lam));
        cpx<float> mrow[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            mrow[k] = a[k] + cdef * (v * conj(vv[k]));
            if (k == r && live) mrow[k].x -= lam;
        }
        gj_invert<NP, float, cpx<float>, false>(mrow, cbuf, r, n, gmask, 0.f);
        const cpx<float> u = group_matvec<NP, float>(mrow, gv, cbuf, r, gmask);

        // GA = -u v^H (row r), then GC (off the diagonal).
        cpx<float> gc[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) gc[k] = mk<float>(0.f, 0.f) - u * conj(vv[k]);  // GA for now
        if (!res.evd) {
            float R[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) R[k] = gc[k].x * crow[k].x + gc[k].y * crow[k].y;  // Re(conj(GA) C)
            // T = G^-1 R (row r): sum_j gi[j] R_j.
            publish<NP, float>(R, fmat, r, gmask);
            float T[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) T[k] = 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j)
#pragma unroll
                for (int k = 0; k < NP; ++k) T[k] += gi[j] * fmat[j * NP + k];
            // GG = -T G^-1 (row r): -sum_j T[j] Ginv_j.
            publish<NP, float>(gi, fmat, r, gmask);
            float GG[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) GG[k] = 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j)
#pragma unroll
                for (int k = 0; k < NP; ++k) GG[k] -= T[j] * fmat[j * NP + k];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float cm2 = norm2(crow[k]);
                const cpx<float> ph = cm2 > 0.f ? rsqrtf(cm2) * crow[k] : mk<float>(0.f, 0.f);
                gc[k] = gi[k] * gc[k] + ((1.f - q.beta) * GG[k]) * ph;
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k)
            if (k == r || k >= n || !live) gc[k] = mk<float>(0.f, 0.f);

        // C -> S.
        const float sr = live ? __ldg(Sd + p * n + r) : 0.f;
        const float rsr = sr > 0.f ? rsqrtf(sr) : 0.f;
        float rs[NP];
        rbuf[r] = rsr;
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < NP; ++k) rs[k] = rbuf[k];
        __syncwarp(gmask);
        float P[NP];
        float rowsum = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            P[k] = gc[k].x * crow[k].x + gc[k].y * crow[k].y;
            rowsum += P[k];
        }
        publish<NP, float>(P, fmat, r, gmask);
        float colsum = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) colsum += fmat[i * NP + r];
        cpx<float> gs[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) gs[k] = (rsr * rs[k]) * gc[k];
        if (live && sr > 0.f) gs[r] = mk<float>(-(rowsum + colsum) / (2.f * sr), 0.f);

        // H = GS + GS^H, packed upper triangle.
        publish<NP, cpx<float>>(gs, cmat, r, gmask);
        if (live) {
            float2 *Hp = Hout + p * nt;
#pragma unroll
            for (int k = 0; k < NP; ++k)
                if (k >= r && k < n) {
                    const cpx<float> h = gs[k] + conj(cmat[k * NP + r]);
                    Hp[packed_index(n, r, k)] = make_float2(h.x, h.y);
                }
        }
        __syncwarp(gmask);
    }
}

// First-order phase uncertainty: white circular noise of variance sigma2 on
// every SLC sample, E|n|^2 = sigma2, propagated through the linked phases.
// With g(q) = H_p z(q) the gradient of phihat_i(p) over the pixel's masked
// window, Var phihat_i = (sigma2 / 2) sum_q |g(q)|^2 = (sigma2 / 2) tr(H^H H S),
// S = sum_q m(q) z(q) z(q)^H, S_jk = C_jk sqrt(S_jj S_kk).  H is Hermitian, so
// tr(H^H H S) = sum_k <row k of H, row k of H S>: each lane's own rows.
// One pass per date with the weight e_i; the reference date has 0.  One warp
// a CTA (the shared buffers of a 32-lane group take 30 KB).
constexpr int kUncWarps = 1;

template <int NP>
__global__ void __launch_bounds__(kUncWarps * 32) k_adj_uncert(const float2 *__restrict__ C,
                                                               const float *__restrict__ Sd, int n, long long npx,
                                                               int ref, const EmiParams prm, float sigma2,
                                                               float *__restrict__ sd_out) {
    constexpr bool kPow2 = (NP & (NP - 1)) == 0;
    constexpr int G = kPow2 ? 32 / NP : 1;
    constexpr int kRowPitch = NP + 2;
    constexpr int kGrpBuf = 2 * NP + 2;
    __shared__ __align__(16) cpx<float> sbuf[kUncWarps][G * kGrpBuf];
    __shared__ __align__(16) cpx<float> rowcache[kUncWarps * 32 * kRowPitch];
    __shared__ __align__(16) cpx<float> mats[kUncWarps][32 * NP];
    __shared__ __align__(16) cpx<float> smats[kUncWarps][32 * NP];  // S of the group's pixel
    __shared__ __align__(16) float ginvs[kUncWarps][32 * NP];       // G^-1 of the group's pixel
    __shared__ __align__(16) cpx<float> vs[kUncWarps][32];
    __shared__ __align__(16) float rss[kUncWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = kPow2 ? lane / NP : 0, r = lane - grp * NP;  // 24-entry rows: one pixel a warp
    const int glane0 = grp * NP;
    const unsigned gmask = (NP >= 24) ? 0xffffffffu : (((1u << NP) - 1u) << glane0);
    const long long nt = ntri(n);
    const long long step = (long long)gridDim.x * kUncWarps * G;
    cpx<float> *myrow = rowcache + (size_t)(warp * 32 + lane) * kRowPitch;
    cpx<float> *cbuf = &sbuf[warp][grp * kGrpBuf];
    cpx<float> *cmat = &mats[warp][grp * NP * NP];
    cpx<float> *smat = &smats[warp][grp * NP * NP];
    const UncShared<NP> sh{myrow, &vs[warp][glane0], &rss[warp][glane0], &ginvs[warp][grp * NP * NP]};
    EmiParams q = prm;
    q.fp64_resolve = 0;
    const float qnan = __int_as_float(0x7fc00000);

    for (long long base = ((long long)blockIdx.x * kUncWarps + warp) * G; base < npx; base += step) {
        const long long p = base + grp;
        const bool valid = p < npx;
        const float2 *Cpix = C + (valid ? p : 0) * nt;
        const bool live = r < n;
        bool nan = false;
        if (valid && live) nan = isnan(__ldg(Cpix + packed_index(n, r, r)).x);
        nan = __any_sync(gmask, nan);
        if (!valid) continue;
        if (nan) {
            if (live) sd_out[(long long)r * npx + p] = qnan;
            continue;
        }
        adj_load_row<NP>(myrow, Cpix, r, n);
        __syncwarp(gmask);
        AdjPixelState<NP> S;
        adj_prepare<NP>(S, sh, Sd, p, r, n, ref, q, cbuf, gmask, glane0);
        // S rows (unnormalised): S_rk = C_rk sqrt(S_rr S_kk)
        {
            // sqrt(S_rr S_kk) = sqrt(S_rr) / rs_k, rs_k = 1 / sqrt(S_kk) (0 where S_kk = 0)
            const float sq_r = sqrtf(S.sr);
            cpx<float> srow[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float rk = sh.rsg[k];
                srow[k] = (live && k < n && rk > 0.f) ? (sq_r / rk) * myrow[k] : mk<float>(0.f, 0.f);
            }
            publish<NP, cpx<float>>(srow, smat, r, gmask);
        }
        float sd_mine = 0.f;  // this lane's date
        for (int i = 0; i < n; ++i) {
            if (i == ref) continue;  // uniform across the group
            cpx<float> h[NP];
            adj_h_row<NP>(S, sh, (r == i) ? 1.f : 0.f, r, n, ref, q.beta, cbuf, cmat, gmask, h);
            // row r of M = H S, then <row r of H, row r of M>
            float tr = 0.f;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                if (k >= n) break;  // S and H are zero past n
                cpx<float> m = mk<float>(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    if (j >= n) break;
                    m = cfma(h[j], smat[j * NP + k], m);
                }
                tr += h[k].x * m.x + h[k].y * m.y;  // Re(conj(h_k) m_k)
            }
            tr = group_sum<NP, float>(live ? tr : 0.f, gmask);
            if (r == i) sd_mine = sqrtf(fmaxf(0.5f * sigma2 * tr, 0.f));
        }
        if (live) sd_out[(long long)r * npx + p] = sd_mine;  // 0 at the reference date
        __syncwarp(gmask);
    }
}

// Per (input pixel q, date i): g_i(q) = sum over the output pixels p whose
// window holds q, with q's mask bit set, of sum_k H_p,ik z_k(q).  NT >= n.
// The date index runs fastest across threads: a warp covers one or two
// pixels, so its loads of H_p rows fall on one or two packed matrices and the
// loads of z(q) are broadcasts.
template <int NT>
__global__ void __launch_bounds__(256) k_adj_gather(const __grid_constant__ Planes z, int n, const Geom g,
                                                    const uint64_t *__restrict__ mask,
                                                    const float2 *__restrict__ H, float2 *__restrict__ grad) {
    const long long npix = (long long)g.H * g.W;
    const long long total = npix * n;
    const long long nt = ntri(n);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long qi = t / n;
        const int i = (int)(t - qi * n);
        const int qy = (int)(qi / g.W), qx = (int)(qi - (long long)qy * g.W);
        cpx<float> zq[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            const float2 v = k < n ? __ldg(z.p[k] + qi) : make_float2(0.f, 0.f);
            zq[k] = mk<float>(v.x, v.y);
        }
        // output rows/columns whose window centre lies within hy/hx of q
        const int oy_lo = max(0, (qy - g.hy - g.sy / 2 + g.sy - 1) / g.sy);
        const int oy_hi = min(g.Ho - 1, (qy + g.hy - g.sy / 2) >= 0 ? (qy + g.hy - g.sy / 2) / g.sy : -1);
        const int ox_lo = max(0, (qx - g.hx - g.sx / 2 + g.sx - 1) / g.sx);
        const int ox_hi = min(g.Wo - 1, (qx + g.hx - g.sx / 2) >= 0 ? (qx + g.hx - g.sx / 2) / g.sx : -1);
        cpx<float> acc = mk<float>(0.f, 0.f);
        for (int oy = oy_lo; oy <= oy_hi; ++oy) {
            const int dy = qy - (oy * g.sy + g.sy / 2);
            if (dy < -g.hy || dy > g.hy) continue;
            for (int ox = ox_lo; ox <= ox_hi; ++ox) {
                const int dx = qx - (ox * g.sx + g.sx / 2);
                if (dx < -g.hx || dx > g.hx) continue;
                const long long o = (long long)oy * g.Wo + ox;
                const int b = (dy + g.hy) * g.wx + (dx + g.hx);
                if (!((__ldg(mask + o * g.nwords + (b >> 6)) >> (b & 63)) & 1ull)) continue;
                const float2 *Hp = H + o * nt;
#pragma unroll
                for (int k = 0; k < NT; ++k) {
                    if (k >= n) break;
                    // H_ik from the packed upper triangle (H Hermitian)
                    const float2 h = __ldg(Hp + (i <= k ? packed_index(n, i, k) : packed_index(n, k, i)));
                    const cpx<float> hik = i <= k ? mk<float>(h.x, h.y) : mk<float>(h.x, -h.y);
                    acc = cfma(hik, zq[k], acc);
                }
            }
        }
        grad[(long long)i * npix + qi] = make_float2(acc.x, acc.y);
    }
}

// Gradient of L with respect to real per-sample window weights (the SHP mask
// read as weights w_b in S = sum_b w_b z(q_b) z(q_b)^H, evaluated at w = mask):
// dL/dw_b = Re sum_jk conj(GS_jk) z_j conj(z_k) = (1/2) z^H H_p z, z = z(q_b);
// 0 for window samples outside the image and for pixels without data (H_p = 0).
// One thread per (output pixel, window sample), samples fastest: a warp spans
// one or two pixels, so its loads of H_p are broadcasts.  NT >= n.
template <int NT>
__global__ void __launch_bounds__(256) k_adj_wgrad(const __grid_constant__ Planes z, int n, const Geom g,
                                                   const float2 *__restrict__ H, float *__restrict__ dw) {
    const long long npx = (long long)g.Ho * g.Wo;
    const int nb = g.wy * g.wx;
    const long long total = npx * nb;
    const long long nt = ntri(n);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long o = t / nb;
        const int b = (int)(t - o * nb);
        const int oy = (int)(o / g.Wo), ox = (int)(o - (long long)oy * g.Wo);
        const int by = b / g.wx, bx = b - by * g.wx;
        const int y = oy * g.sy + g.sy / 2 - g.hy + by, x = ox * g.sx + g.sx / 2 - g.hx + bx;
        float acc = 0.f;
        if (y >= 0 && y < g.H && x >= 0 && x < g.W) {
            const long long qi = (long long)y * g.W + x;
            cpx<float> zq[NT];
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                const float2 v = k < n ? __ldg(z.p[k] + qi) : make_float2(0.f, 0.f);
                zq[k] = mk<float>(v.x, v.y);
            }
            // z^H H z = sum_j H_jj |z_j|^2 + 2 Re sum_{j<k} conj(z_j) H_jk z_k
            const float2 *Hp = H + o * nt;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (j >= n) break;
                const float2 *row = Hp + packed_index(n, j, j);
                const float2 hd = __ldg(row);
                cpx<float> s = mk<float>(0.f, 0.f);
#pragma unroll
                for (int k = j + 1; k < NT; ++k) {
                    if (k >= n) break;
                    const float2 h = __ldg(row + (k - j));
                    s = cfma(mk<float>(h.x, h.y), zq[k], s);
                }
                acc += hd.x * norm2(zq[j]) + 2.f * (zq[j].x * s.x + zq[j].y * s.y);
            }
        }
        dw[t] = 0.5f * acc;
    }
}

// Tiled scatter of the same sum: a CTA owns a TY x TX tile of output pixels,
// stages the z of the input region their windows cover and a region-sized
// accumulator in shared memory; item (pixel s, row i) loads row i of H_p once
// and adds (H_p z(q))_i into the accumulator for every accepted look q; the
// accumulator is then added into the gradient (tiles overlap by the window
// halo).  H is read once; the sums are shared-memory atomics, so the order of
// additions (and the last bits of the result) may vary from run to run.
struct AdjTile {
    int TY, TX, RY, RX, L;
};

template <int NT>
__global__ void __launch_bounds__(256) k_adj_scatter(const __grid_constant__ Planes z, int n, const Geom g,
                                                     const uint64_t *__restrict__ mask, const float2 *__restrict__ H,
                                                     float2 *__restrict__ grad, const AdjTile t, long long ntiles,
                                                     int tilesY) {
    extern __shared__ __align__(16) float2 sm[];
    const int npr = t.RY * t.RX;
    float2 *zreg = sm;                                         // [npr][n]
    float2 *acc = sm + (size_t)npr * n;                        // [npr][n]
    int *lkoff = reinterpret_cast<int *>(acc + (size_t)npr * n);  // [L]
    const long long nt = ntri(n);
    const long long npix = (long long)g.H * g.W;
    for (int l = threadIdx.x; l < t.L; l += blockDim.x) lkoff[l] = (l / g.wx) * t.RX + (l % g.wx);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ty0 = (int)(tile % tilesY) * t.TY, tx0 = (int)(tile / tilesY) * t.TX;
        const int y0 = ty0 * g.sy + g.sy / 2 - g.hy, x0 = tx0 * g.sx + g.sx / 2 - g.hx;
        __syncthreads();  // previous tile done with the buffers (and the look table written)
        for (int idx = threadIdx.x; idx < npr * n; idx += blockDim.x) {
            const int d = idx / npr, pr = idx - d * npr;
            const int y = y0 + pr / t.RX, x = x0 + pr % t.RX;
            float2 v = make_float2(0.f, 0.f);
            if (y >= 0 && y < g.H && x >= 0 && x < g.W) v = __ldg(z.p[d] + (long long)y * g.W + x);
            zreg[pr * n + d] = v;
            acc[pr * n + d] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int items = t.TY * t.TX * n;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int s = it / n, i = it - s * n;
            const int tx = s / t.TY, ty = s - tx * t.TY;
            const int oy = ty0 + ty, ox = tx0 + tx;
            if (oy >= g.Ho || ox >= g.Wo) continue;
            const long long o = (long long)oy * g.Wo + ox;
            const float2 *Hp = H + o * nt;
            cpx<float> hrow[NT];
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                hrow[k] = mk<float>(0.f, 0.f);
                if (k < n) {
                    const float2 h = __ldg(Hp + (i <= k ? packed_index(n, i, k) : packed_index(n, k, i)));
                    hrow[k] = i <= k ? mk<float>(h.x, h.y) : mk<float>(h.x, -h.y);
                }
            }
            const uint64_t *mw = mask + o * g.nwords;
            const int corner = ty * g.sy * t.RX + tx * g.sx;
            for (int w0 = 0; w0 < t.L; w0 += 64) {
                uint64_t bits = __ldg(mw + (w0 >> 6));
                if (t.L - w0 < 64) bits &= (1ull << (t.L - w0)) - 1ull;  // only the window's looks
                while (bits) {
                    const int l = w0 + __ffsll((long long)bits) - 1;
                    bits &= bits - 1;
                    const float2 *zq = zreg + (size_t)(corner + lkoff[l]) * n;
                    cpx<float> a = mk<float>(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < NT; ++k) {
                        if (k >= n) break;
                        const float2 zz = zq[k];
                        a = cfma(hrow[k], mk<float>(zz.x, zz.y), a);
                    }
                    float2 *dst = acc + (size_t)(corner + lkoff[l]) * n + i;
                    atomicAdd(&dst->x, a.x);
                    atomicAdd(&dst->y, a.y);
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < npr * n; idx += blockDim.x) {
            const int d = idx / npr, pr = idx - d * npr;
            const int y = y0 + pr / t.RX, x = x0 + pr % t.RX;
            if (y < 0 || y >= g.H || x < 0 || x >= g.W) continue;
            const float2 v = acc[pr * n + d];
            if (v.x == 0.f && v.y == 0.f) continue;
            float2 *dst = grad + (long long)d * npix + (long long)y * g.W + x;
            atomicAdd(&dst->x, v.x);
            atomicAdd(&dst->y, v.y);
        }
    }
}

// Tile for the scatter: the most output pixels whose region (z and
// accumulator, n samples each) fits the budget.
static AdjTile adj_tile(int n, const Geom &g, size_t budget) {
    AdjTile best{0, 0, 0, 0, g.wy * g.wx};
    for (int TY = 1; TY <= 32; ++TY)
        for (int TX = 1; TX <= 64; ++TX) {
            AdjTile c{TY, TX, (TY - 1) * g.sy + g.wy, (TX - 1) * g.sx + g.wx, g.wy * g.wx};
            const size_t sm = (size_t)c.RY * c.RX * n * 2 * sizeof(float2) + (size_t)c.L * sizeof(int);
            if (sm > budget) continue;
            if (TY * TX > best.TY * best.TX ||
                (TY * TX == best.TY * best.TX && c.RY * c.RX < best.RY * best.RX))
                best = c;
        }
    return best;
}

static int adj_grid(long long work) {
    long long blocks = (work + 255) / 256;
    const long long cap = (long long)device_sm_count() * 8;
    return (int)std::max<long long>(1, std::min(blocks, cap));
}

template <int NP>
static cudaError_t run_adj_pixel(const float2 *C, const float *Sd, int n, long long npx, int ref,
                                 const EmiParams &prm, const float *w, float2 *H, cudaStream_t s) {
    constexpr int G = (NP & (NP - 1)) ? 1 : 32 / NP;
    long long blocks = ((npx + G - 1) / G + kAdjWarps - 1) / kAdjWarps;
    const long long cap = (long long)device_sm_count() * 16;
    blocks = std::max<long long>(1, std::min(blocks, cap));
    k_adj_pixel<NP><<<(unsigned)blocks, kAdjWarps * 32, 0, s>>>(C, Sd, n, npx, ref, prm, w, H);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t run_adj_uncert(const float2 *C, const float *Sd, int n, long long npx, int ref,
                                  const EmiParams &prm, float sigma2, float *out, cudaStream_t s) {
    constexpr int G = (NP & (NP - 1)) ? 1 : 32 / NP;
    long long blocks = ((npx + G - 1) / G + kUncWarps - 1) / kUncWarps;
    const long long cap = (long long)device_sm_count() * 32;
    blocks = std::max<long long>(1, std::min(blocks, cap));
    k_adj_uncert<NP><<<(unsigned)blocks, kUncWarps * 32, 0, s>>>(C, Sd, n, npx, ref, prm, sigma2, out);
    return cudaGetLastError();
}

// Workspace layout: C [npx][ntri], H [npx][ntri], Sd [npx][n] (256-byte aligned parts).
size_t adjoint_workspace_bytes(int n, const Geom &g) {
    const long long npx = (long long)g.Ho * g.Wo;
    auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return 2 * a256((size_t)npx * ntri(n) * sizeof(float2)) + a256((size_t)npx * n * sizeof(float));
}

// Recomputed coherence, diagonal sums and H_p of every output pixel into the
// workspace; *Hout points at H.  npx > 0.
static cudaError_t adjoint_h(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                             const EmiParams &prm, const float *dphase, void *workspace, cudaStream_t s, Prof *prof,
                             float2 **Hout) {
    const long long npx = (long long)g.Ho * g.Wo;
    auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *ws = static_cast<char *>(workspace);
    float2 *C = reinterpret_cast<float2 *>(ws);
    float2 *H = reinterpret_cast<float2 *>(ws + a256((size_t)npx * ntri(n) * sizeof(float2)));
    float *Sd = reinterpret_cast<float *>(ws + 2 * a256((size_t)npx * ntri(n) * sizeof(float2)));
    *Hout = H;
    if (prof) prof->begin("adjoint_covariance", s);
    cudaError_t e = launch_covariance(z, n, g, mask, C, s);  // recomputed, not stored by the forward pass
    if (prof) prof->end(s);
    if (e != cudaSuccess) return e;
    if (prof) prof->begin("adjoint_pixel", s);
    k_adj_sdiag<<<adj_grid(npx * n), 256, 0, s>>>(z, n, g, mask, Sd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n <= 8) e = run_adj_pixel<8>(C, Sd, n, npx, ref, prm, dphase, H, s);
    else if (n <= 16) e = run_adj_pixel<16>(C, Sd, n, npx, ref, prm, dphase, H, s);
    else if (n <= 24) e = run_adj_pixel<24>(C, Sd, n, npx, ref, prm, dphase, H, s);
    else e = run_adj_pixel<32>(C, Sd, n, npx, ref, prm, dphase, H, s);
    if (prof) prof->end(s);
    return e;
}

cudaError_t launch_adjoint(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                           const EmiParams &prm, const float *dphase, void *workspace, float2 *grad,
                           cudaStream_t s, Prof *prof) {
    const long long npx = (long long)g.Ho * g.Wo, npix = (long long)g.H * g.W;
    if (npx == 0) return cudaMemsetAsync(grad, 0, (size_t)npix * n * sizeof(float2), s);
    float2 *H = nullptr;
    cudaError_t e = adjoint_h(z, n, g, mask, ref, prm, dphase, workspace, s, prof, &H);
    if (e != cudaSuccess) return e;
    if (prof) prof->begin("adjoint_gather", s);
    const size_t kBudget = 150 * 1024;
    const AdjTile t = adj_tile(n, g, kBudget);
    if (t.TY > 0) {
        // tiled scatter (H read once)
        const size_t smem = (size_t)t.RY * t.RX * n * 2 * sizeof(float2) + (size_t)t.L * sizeof(int);
        e = cudaMemsetAsync(grad, 0, (size_t)npix * n * sizeof(float2), s);
        if (e != cudaSuccess) return e;
        const int tilesY = (g.Ho + t.TY - 1) / t.TY;
        const long long ntiles = (long long)tilesY * ((g.Wo + t.TX - 1) / t.TX);
        const long long gridT = std::min<long long>(ntiles, (long long)device_sm_count() * 2);
        if (n <= 8) {
            cudaFuncSetAttribute(k_adj_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);
            k_adj_scatter<8><<<(unsigned)gridT, 256, smem, s>>>(z, n, g, mask, H, grad, t, ntiles, tilesY);
        } else if (n <= 16) {
            cudaFuncSetAttribute(k_adj_scatter<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);
            k_adj_scatter<16><<<(unsigned)gridT, 256, smem, s>>>(z, n, g, mask, H, grad, t, ntiles, tilesY);
        } else {
            cudaFuncSetAttribute(k_adj_scatter<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);
            k_adj_scatter<32><<<(unsigned)gridT, 256, smem, s>>>(z, n, g, mask, H, grad, t, ntiles, tilesY);
        }
    } else {
        // window too large for a shared-memory region: per-element gather
        const int grid = adj_grid(npix * n);
        if (n <= 8) k_adj_gather<8><<<grid, 256, 0, s>>>(z, n, g, mask, H, grad);
        else if (n <= 16) k_adj_gather<16><<<grid, 256, 0, s>>>(z, n, g, mask, H, grad);
        else k_adj_gather<32><<<grid, 256, 0, s>>>(z, n, g, mask, H, grad);
    }
    e = cudaGetLastError();
    if (prof) prof->end(s);
    return e;
}

// Gradient of L = sum(dphase * phase) with respect to the window weights
// [Ho][Wo][wy*wx] (k_adj_wgrad) over the workspace of the adjoint.
cudaError_t launch_weight_gradient(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                                   const EmiParams &prm, const float *dphase, void *workspace, float *dw,
                                   cudaStream_t s) {
    const long long npx = (long long)g.Ho * g.Wo;
    if (npx == 0) return cudaSuccess;
    float2 *H = nullptr;
    cudaError_t e = adjoint_h(z, n, g, mask, ref, prm, dphase, workspace, s, nullptr, &H);
    if (e != cudaSuccess) return e;
    const int grid = adj_grid(npx * g.wy * g.wx);
    if (n <= 8) k_adj_wgrad<8><<<grid, 256, 0, s>>>(z, n, g, H, dw);
    else if (n <= 16) k_adj_wgrad<16><<<grid, 256, 0, s>>>(z, n, g, H, dw);
    else k_adj_wgrad<32><<<grid, 256, 0, s>>>(z, n, g, H, dw);
    return cudaGetLastError();
}

// First-order phase standard deviations (k_adj_uncert) over the workspace of
// the adjoint: the coherence and the diagonal sums are recomputed there.
cudaError_t launch_phase_uncertainty(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                                     const EmiParams &prm, float sigma2, void *workspace, float *sd,
                                     cudaStream_t s) {
    const long long npx = (long long)g.Ho * g.Wo;
    if (npx == 0) return cudaSuccess;
    auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *ws = static_cast<char *>(workspace);
    float2 *C = reinterpret_cast<float2 *>(ws);
    float *Sd = reinterpret_cast<float *>(ws + 2 * a256((size_t)npx * ntri(n) * sizeof(float2)));
    cudaError_t e = launch_covariance(z, n, g, mask, C, s);
    if (e != cudaSuccess) return e;
    k_adj_sdiag<<<adj_grid(npx * n), 256, 0, s>>>(z, n, g, mask, Sd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n <= 8) return run_adj_uncert<8>(C, Sd, n, npx, ref, prm, sigma2, sd, s);
    if (n <= 16) return run_adj_uncert<16>(C, Sd, n, npx, ref, prm, sigma2, sd, s);
    if (n <= 24) return run_adj_uncert<24>(C, Sd, n, npx, ref, prm, sigma2, sd, s);
    return run_adj_uncert<32>(C, Sd, n, npx, ref, prm, sigma2, sd, s);
}

}  // namespace plk
