// S4-S6 device routines: EMI phase linking (Sec. III-B, eq.
// (emi-eigenvalue-problem)), the reference phase (Sec. II-A) and the temporal
// coherence (Sec. III-C, eq. (temporal-coherence)) of one pixel.
//
// A pixel is served by a group of NP lanes (NP = 8, 16, 20, 24, 28 or 32 >= N,
// the last four one pixel a warp); lane r owns row r of every N x N matrix,
// held in registers.  Padded rows/columns
// (r >= N) carry the identity and are never touched by the elimination steps.
// Row broadcasts go through a per-group shared-memory buffer read with
// 16-byte loads (one wavefront serves the whole group); reductions are
// xor-butterflies inside the group, which leave bit-identical sums in every
// lane, so loop exits stay group-uniform.
//
//   G   = (1 - beta)|C| + beta I, inverted in place by Gauss-Jordan without
//         pivoting (for symmetric positive definite G its pivots are the
//         squared Cholesky pivots).
//   B   = G^{-1} o C - mu I, inverted the same way in complex arithmetic.
//   v   = lim x_{t+1} = B^{-1} x_t / |B^{-1} x_t| (inverse iteration with
//         shift mu = 0.99, Sec. III-B), started from the phases of column 0
//         of C.
//   EVD fallback where G is not invertible: the largest eigenvector of C
//         (Sec. III-B), by power iteration, refined by shifted inverse
//         iteration on -C when that converges slowly.
#pragma once

#include "cpx.cuh"
#include "plk_internal.cuh"

namespace plk {

template <class T> struct Lim;
template <> struct Lim<float> {
    static constexpr float tiny = 1e-30f;
    static constexpr float big = 3.0e38f;
};
template <> struct Lim<double> {
    static constexpr double tiny = 1e-300;
    static constexpr double big = 1e300;
};

// The inversion of G fails (EVD fallback, Sec. III-B) when its Cholesky
// factorisation meets a pivot <= kPivotFail (G has unit diagonal): G is
// indefinite, as |C| of a highly coherent C often is, or too close to
// singular.  The Gauss-Jordan pivots are the same Schur complements.  In
// single precision a pivot within kPivotBand of the limit is left to the
// double-precision path (about 0.05% of pixels on burst-shaped stacks).
constexpr double kPivotFail = 1e-4;
constexpr double kPivotBand = 2e-5;

// Lanes a group's reductions span: NP when it is a power of two; otherwise
// (rows of 20, 24 or 28 entries) the whole warp, one pixel a warp, the lanes past the
// last row contributing the reduction's identity (their rows are all zero, and
// every caller passes 0, or the identity, for rows past n).
template <int NP>
struct GroupLanes {
    static constexpr int value = (NP & (NP - 1)) ? 32 : NP;
};

template <int NP, class T>
__device__ __forceinline__ T group_sum(T v, unsigned gmask) {
#pragma unroll
    for (int off = GroupLanes<NP>::value / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(gmask, v, off);
    return v;
}
template <int NP, class T>
__device__ __forceinline__ T group_max(T v, unsigned gmask) {
#pragma unroll
    for (int off = GroupLanes<NP>::value / 2; off >= 1; off >>= 1) v = fmax(v, __shfl_xor_sync(gmask, v, off));
    return v;
}
template <int NP, class T>
__device__ __forceinline__ T group_min(T v, unsigned gmask) {
#pragma unroll
    for (int off = GroupLanes<NP>::value / 2; off >= 1; off >>= 1) v = fmin(v, __shfl_xor_sync(gmask, v, off));
    return v;
}

// ---- scalar helpers over real T and complex cpx<T> -----------------------
__device__ __forceinline__ float inv_s(float a) { return 1.0f / a; }
__device__ __forceinline__ double inv_s(double a) { return 1.0 / a; }
template <class T>
__device__ __forceinline__ cpx<T> inv_s(cpx<T> a) {
    const T d = T(1) / norm2(a);
    return mk<T>(a.x * d, -a.y * d);
}
__device__ __forceinline__ float mul_s(float a, float b) { return a * b; }
__device__ __forceinline__ double mul_s(double a, double b) { return a * b; }
template <class T>
__device__ __forceinline__ cpx<T> mul_s(cpx<T> a, cpx<T> b) { return a * b; }
__device__ __forceinline__ float fms_s(float a, float b, float c) { return c - a * b; }
__device__ __forceinline__ double fms_s(double a, double b, double c) { return c - a * b; }
template <class T>
__device__ __forceinline__ cpx<T> fms_s(cpx<T> a, cpx<T> b, cpx<T> c) { return cfms(a, b, c); }
// |c| from |c|^2: x * rsqrt(x) in single precision (a few ulp, one MUFU
// operation instead of a correctly rounded square root), sqrt in double.
__device__ __forceinline__ float mag_t(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }
__device__ __forceinline__ double mag_t(double v) { return sqrt(v); }
// Reciprocal of a pivot: one approximate MUFU operation in single precision
// (rcp.approx, at most 1 ulp off), a division in double precision.
__device__ __forceinline__ float rcp_t(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
// Double: the single-precision seed refined by two Newton steps
// r <- r + r (1 - a r), each squaring the relative error (2^-23 -> 2^-46 ->
// rounding level); outside the single-precision range, a division.
__device__ __forceinline__ double rcp_t(double a) {
    const double m = fabs(a);
    if (!(m > 1e-30 && m < 1e30)) return 1.0 / a;
    double r = (double)rcp_t((float)a);
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ float scale_s(float a, float s) { return a * s; }
__device__ __forceinline__ double scale_s(double a, double s) { return a * s; }
template <class T>
__device__ __forceinline__ cpx<T> scale_s(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
__device__ __forceinline__ float neg_s(float a) { return -a; }
__device__ __forceinline__ double neg_s(double a) { return -a; }
template <class T>
__device__ __forceinline__ cpx<T> neg_s(cpx<T> a) { return mk<T>(-a.x, -a.y); }
__device__ __forceinline__ float re_s(float a) { return a; }
__device__ __forceinline__ double re_s(double a) { return a; }
template <class T>
__device__ __forceinline__ T re_s(cpx<T> a) { return a.x; }
__device__ __forceinline__ float real_s(float, float v) { return v; }
__device__ __forceinline__ double real_s(double, double v) { return v; }
template <class T>
__device__ __forceinline__ cpx<T> real_s(cpx<T>, T v) { return mk<T>(v, T(0)); }

// In-place Gauss-Jordan inverse (no pivoting) of the matrix whose row r is
// held by lane r of the group.  The step loop is not unrolled, so the pivot
// column cannot be a runtime register index; instead each lane keeps its row
// rotated: at step k, a[c] holds column (k + c) mod NP, so the pivot column is
// always a[0].  Step k: lane k publishes its row as it stands; every lane
// reads it, takes the pivot p = row[0], and with f' = a[0]/p updates
//     a[c-1] <- a[c] - f' row[c]   (c = 1..NP-1),   a[NP-1] <- -f'
// shifting its row one place left; the pivot lane uses f' = 1 - 1/p, which
// turns the same update into row[c]/p, and takes 1/p as its new last entry.
// After NP steps the rotation is complete and a[c] holds column c of the
// inverse.  Padded rows/columns (index >= n) are the identity: their steps have
// pivot 1 and f' = 0 on every lane, so they only rotate the rows (no publish,
// no arithmetic).  The pivot is taken as the real part of row[0] (the matrices
// inverted here are real symmetric or Hermitian).  The pivot lane's update can
// lose relative accuracy ~eps*|p| for pivots far above 1 (the complex B only,
// whose inverse serves as a preconditioner); G has pivots <= 1.
// PD = true (real G): a pivot <= tiny is replaced by tiny.  PD = false
// (complex B, possibly indefinite): only a pivot of magnitude below tiny is.
// Every lane sees every pivot, so all return the same value: the first real
// pivot (in step order, over the first n steps, before replacement) that is
// <= thr -- the one a Cholesky factorisation would stop at -- or, if there is
// none, the smallest pivot.
// a[c] <- a[(c + s) mod NP] for a group-uniform 0 <= s < NP.  Rows of 8 and
// 16 entries: one conditional rotation per bit of s (NP moves each) instead of
// s single-place shifts.  Rows beyond 16 entries (one pixel a warp, few padded
// pivots): single-place shifts in a loop, short code, measured 12% faster at
// N = 20 and 28 than conditional rotations, which are long code even where
// they move nothing.
template <int NP, class S>
__device__ __forceinline__ void rotate_left(S (&a)[NP], int s) {
    if constexpr (NP > 16) {
#pragma unroll 1
        for (int t = 0; t < s; ++t) {
            const S t0 = a[0];
#pragma unroll
            for (int j = 0; j + 1 < NP; ++j) a[j] = a[j + 1];
            a[NP - 1] = t0;
        }
    } else {
        static_assert((NP & (NP - 1)) == 0, "rows of up to 16 entries are 8 or 16");
#pragma unroll
        for (int b = NP / 2; b >= 1; b >>= 1) {
            if (s & b) {
                // b cycles of NP / b entries, one temporary each
#pragma unroll
                for (int c = 0; c < b; ++c) {
                    const S t = a[c];
#pragma unroll
                    for (int i = 0; i + 1 < NP / b; ++i) a[c + i * b] = a[c + (i + 1) * b];
                    a[c + NP - b] = t;
                }
            }
        }
    }
}

template <int NP, class T, class S, bool PD>
__device__ __forceinline__ T gj_invert(S (&a)[NP], S *buf, int r, int n, unsigned gmask, T thr) {
    constexpr int E = 16 / sizeof(S);
    static_assert(NP % E == 0, "row must be a multiple of 16 bytes");
    T minpiv = Lim<T>::big;
    T first_low = Lim<T>::big;
    bool have_low = false;
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        const bool pivot_lane = (r == k);
        if (pivot_lane) {
            uint4 *dst = reinterpret_cast<uint4 *>(buf);
#pragma unroll
            for (int q = 0; q < NP / E; ++q) {
                uint4 v;
                memcpy(&v, &a[q * E], 16);
                dst[q] = v;
            }
        }
        __syncwarp(gmask);
        const uint4 *src = reinterpret_cast<const uint4 *>(buf);
        T pr;
        {
            const uint4 v0 = src[0];
            S p0[E];
            memcpy(p0, &v0, 16);
            pr = re_s(p0[0]);
        }
        minpiv = fmin(minpiv, pr);
        if (!have_low && pr <= thr) {
            have_low = true;
            first_low = pr;
        }
        // The pivots of a Hermitian matrix are real (Schur complements of a
        // Hermitian matrix are Hermitian); the imaginary part of a computed
        // complex pivot is rounding noise and is dropped.
        if (PD) {
            if (!(pr > Lim<T>::tiny)) pr = Lim<T>::tiny;
        } else {
            if (!(abs_t(pr) > Lim<T>::tiny)) pr = Lim<T>::tiny;
        }
        const T inv = rcp_t(pr);
        const S fp = pivot_lane ? real_s(a[0], T(1) - inv) : scale_s(a[0], inv);
#pragma unroll
        for (int q = 0; q < NP / E; ++q) {
            const uint4 v = src[q];
            S p[E];
            memcpy(p, &v, 16);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = q * E + e;
                if (j > 0) a[j - 1] = fms_s(fp, p[e], a[j]);
            }
        }
        a[NP - 1] = pivot_lane ? real_s(a[0], inv) : neg_s(fp);
        __syncwarp(gmask);
    }
    // Padded pivots k >= n (identity row and column): f' = 0 on every lane and
    // the entry rotated in is the one rotated out, so each such step is a
    // rotation by one place; all of them together, a rotation by NP - n.
    rotate_left<NP, S>(a, NP - n);
    return have_low ? first_low : minpiv;
}

// y = sum_j a[j] * v_j where v (one entry per lane) is published in buf.
template <int NP, class T>
__device__ __forceinline__ cpx<T> group_matvec(const cpx<T> (&a)[NP], cpx<T> v, cpx<T> *buf, int r,
                                               unsigned gmask) {
    constexpr int E = 16 / sizeof(cpx<T>);
    buf[r] = v;
    __syncwarp(gmask);
    cpx<T> y = mk<T>(T(0), T(0));
    const uint4 *src = reinterpret_cast<const uint4 *>(buf);
#pragma unroll
    for (int q = 0; q < NP / E; ++q) {
        const uint4 u = src[q];
        cpx<T> xs[E];
        memcpy(xs, &u, 16);
#pragma unroll
        for (int e = 0; e < E; ++e) y = cfma(a[q * E + e], xs[e], y);
    }
    __syncwarp(gmask);
    return y;
}

struct PixelResult {
    float phase;  // this lane's linked phase (row r)
    float tcoh;
    float lam;
    int status;
    bool flag;    // the single-precision solve asks for the FP64 re-solve
    // For the adjoint (single-precision solve): this lane's entry of the unit
    // eigenvector and whether the EVD fallback produced it.
    cpx<float> v;
    bool evd;
};

constexpr int kPending = 0xFE;  // status of a pixel handed to the FP64 re-solve

template <class T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 5.96e-8f; };
template <> struct Eps<double> { static constexpr double v = 1.11e-16; };

// Row source: `load(k)` returns C_rk (complex, unit diagonal) of this lane's
// row for k < n; padded entries are produced here.  A source that already
// holds the padded row (Loader::kPadded) hands it over whole.
template <class L, class = void>
struct IsPadded { static constexpr bool value = false; };
template <class L>
struct IsPadded<L, decltype(void(L::kPadded))> { static constexpr bool value = L::kPadded; };

template <int NP, class T, class Loader>
__device__ __forceinline__ void load_crow(cpx<T> (&c)[NP], const Loader &load, int r, int n) {
    if constexpr (IsPadded<Loader>::value) {
        load.all(c);
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (r < n && k < n) c[k] = load(k);
            else c[k] = mk<T>((k == r) ? T(1) : T(0), T(0));
        }
    }
}

// a <- (G^{-1} o C - mu I)^{-1}, from g = G^{-1} (this lane's row) and C.
// Returns the smallest pivot: by Sylvester's law of inertia the pivots of the
// Hermitian B = A - mu I (the D of its LDL^H factorisation) are all positive
// exactly when B is positive definite, i.e. when mu lies below lambda_min.
template <int NP, class T, class Loader>
__device__ __forceinline__ T form_shift_inverse(cpx<T> (&a)[NP], const T (&g)[NP], const Loader &load, T mu,
                                                cpx<T> *cbuf, int r, int n, unsigned gmask) {
    load_crow<NP, T>(a, load, r, n);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        a[k] = mk<T>(g[k] * a[k].x, g[k] * a[k].y);
        if (k == r) a[k].x -= mu;
    }
    return gj_invert<NP, T, cpx<T>, false>(a, cbuf, r, n, gmask, T(0));
}

// y = A x with A = G^{-1} o C, row r from g and the reloaded C row.
template <int NP, class T, class Loader>
__device__ __forceinline__ cpx<T> apply_A(const T (&g)[NP], const Loader &load, cpx<T> x, cpx<T> *buf, int r,
                                          int n, unsigned gmask) {
    cpx<T> row[NP];
    load_crow<NP, T>(row, load, r, n);
#pragma unroll
    for (int k = 0; k < NP; ++k) row[k] = mk<T>(g[k] * row[k].x, g[k] * row[k].y);
    return group_matvec<NP, T>(row, x, buf, r, gmask);
}

// Inverse iteration x <- B^{-1} x / |B^{-1} x| on the rows a[] (B^{-1}, or C
// itself on the EVD fallback when allow_reshift is false), with the shift
// refinement described at emi_solve: reform(mu) rebuilds a[] for a new shift
// and returns the smallest pivot.  On return d = x^H a x of the last step
// (1/(lambda - mu) for B^{-1}) and q the last convergence factor measured
// above the noise floor.  Returns true on convergence.
//
// floor_num / floor_den (floor_den > 0; 0 = none), a shift below lambda_min(A):
// when B for the starting shift is not positive definite, the shift lies above
// lambda_min and the iteration would converge to the eigenvalue nearest mu
// rather than the smallest one, so the start is rebuilt once at the floor and
// the reshifts move up from there.  For A = G^-1 o C the floor is 0.999 /
// ||G||_inf (lambda_min(G^-1 o C) >= lambda_min(G^-1) min_i C_ii = 1 / lambda_max(G)
// by Schur's bound for a Hadamard product of positive semidefinite matrices);
// for A = -C it is -1.001 ||C||_inf.  The division is taken only when needed.
// *used (when given) receives the number of iteration steps taken, rebuilds
// not counted.  stop_slow (power iteration only): give up as soon as the
// convergence factor is seen to be slow (q > 0.3 after 4 steps), leaving the
// rest of the step budget to the caller's refinement.
template <int NP, class T, class Reform>
__device__ __forceinline__ bool inverse_iteration(cpx<T> (&a)[NP], cpx<T> &x, cpx<T> &d, T &mu, T &q,
                                                  const Reform &reform, bool allow_reshift, cpx<T> *cbuf, int r,
                                                  bool live, unsigned gmask, T tol, int max_iter,
                                                  bool build_first, T floor_num = T(0), T floor_den = T(0),
                                                  int *used = nullptr, bool stop_slow = false) {
    const T tol2 = tol * tol;
    if (used) *used = 0;
    d = mk<T>(T(1), T(0));
    q = T(0);
    T dl_prev = T(-1);
    int in_round = 0, reshifts = 0;
    // reform_to > 0: rebuild a[] for shift mu_try before the next step; a
    // failed inertia check (B not positive definite) rebuilds it once more for
    // the old shift.  One call site keeps the inlined elimination code single.
    T mu_try = mu;
    int pending = build_first ? 2 : 0;  // 0 none, 1 try mu_try, 2 (re)build for mu
    for (int it = 0; it < max_iter + 2 * 3 + 1; ++it) {
        if (pending) {
            const T pmin = reform(pending == 1 ? mu_try : mu);
            if (pending == 1 && pmin > T(0)) {
                mu = mu_try;
                ++reshifts;
                pending = 0;
            } else if (pending == 1) {
                reshifts = 3;
                pending = 2;
                continue;
            } else if (it == 0 && allow_reshift && !(pmin > T(0)) && floor_den > T(0)) {
                // the starting shift is above lambda_min: rebuild below it
                mu = fmin(mu, floor_num / floor_den);
                continue;
            } else {
                pending = 0;
            }
            in_round = 0;
            dl_prev = T(-1);
            q = T(0);
            continue;
        }
        if (it - 2 * reshifts >= max_iter) break;
        if (used) ++*used;
        cpx<T> y = group_matvec<NP, T>(a, x, cbuf, r, gmask);
        if (!live) y = mk<T>(T(0), T(0));
        const T s = group_sum<NP, T>(norm2(y), gmask);          // |y|^2
        d.x = group_sum<NP, T>(x.x * y.x + x.y * y.y, gmask);  // x^H y
        d.y = group_sum<NP, T>(x.x * y.y - x.y * y.x, gmask);
        const T dm2 = norm2(d);
        // Unit iterate with x's common phase: y conj(d) / (|d| |y|).
        const T sc = (s > T(0) && dm2 > T(0)) ? rsqrt_t(s) * rsqrt_t(dm2) : T(0);
        const cpx<T> yn = (sc > T(0)) ? sc * (y * conj(d)) : x;
        const T dl = group_sum<NP, T>(norm2(yn - x), gmask);
        x = yn;
        ++in_round;
        if (dl_prev > T(0) && dl > T(100) * tol2) q = sqrt_t(dl / dl_prev);
        dl_prev = dl;
        if (dl <= tol2) return true;
        if (stop_slow && !allow_reshift && in_round >= 4 && q > T(0.3)) return false;
        if (allow_reshift && reshifts < 3 && in_round >= 4 && q > T(0.3)) {
            // Move the shift towards lambda_min; keep it only if B stays
            // positive definite (the shift is still below lambda_min),
            // otherwise restore the previous one and stop moving it.
            const T lam_est = mu + T(1) / ((d.x != T(0)) ? d.x : Lim<T>::tiny);
            mu_try = mu + T(0.75) * (lam_est - mu);
            pending = 1;
        }
    }
    return false;
}

// Solve one pixel.  T = float: returns flag = true (and no outputs) for a pixel
// whose single-precision result cannot be trusted to err_max, when
// prm.fp64_resolve is set.  T = double: always produces outputs; the inversion
// of G fails (EVD fallback) when a pivot is <= kPivotFail, as in the FP64
// reference.
//
// Shift: inverse iteration starts with mu (0.99, Sec. III-B).  When the
// iterate converges slowly (factor q > 0.3 after 4 steps, i.e. lambda_min sits
// far above mu relative to the gap), the shift moves 3/4 of the way to the
// current eigenvalue estimate mu + 1/(x^H B^{-1} x) (an upper bound of
// lambda_min while B is positive definite) and B^{-1} is rebuilt; at most
// three times.
//
// Error bound: a relative perturbation e of G moves G^{-1} by about
// cond(G) |G^{-1}| e and the eigenvector by that over the eigengap; the gap is
// read off the observed convergence factor q = (l1 - mu)/(l2 - mu).  The bound
// is first order and loose (on synthetic stacks the measured single-precision
// error sits three to four orders of magnitude below it), so pixels are handed
// to double precision when it exceeds err_max (default 0.1).
//
// GSM = true: once inverted, this lane's row of G^{-1} moves to gslot (NP
// values, 16-byte aligned, private to the lane) and is read back where it is
// used -- each rebuild of B^{-1} and the residual correction -- instead of
// holding NP registers through the complex elimination and the iteration.
template <int NP, class T, class Loader, bool GSM = false>
__device__ PixelResult emi_solve(const Loader &load, int r, int n, int ref, const EmiParams &prm,
                                 cpx<T> *cbuf, unsigned gmask, int glane0, bool is_fp64, T *gslot = nullptr) {
    static_assert(!GSM || (NP * sizeof(T)) % 16 == 0, "G^-1 row slot: whole 16-byte chunks");
    PixelResult out;
    out.flag = false;
    T *rbuf = reinterpret_cast<T *>(cbuf);
    const bool live = r < n;

    cpx<T> a[NP];
    load_crow<NP, T>(a, load, r, n);

    // G = (1 - beta)|C| + beta I, and its inverse (kept in g).
    T g[NP];
    T rs = 0, mmin = T(1);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const T mc = mag_t(norm2(a[k]));
        if (k != r && k < n && live) mmin = fmin(mmin, mc);
        T m = mc;
        if (prm.beta != 0.f) m = (T(1) - T(prm.beta)) * m + ((k == r) ? T(prm.beta) : T(0));
        g[k] = m;
        rs += abs_t(m);
    }
    // Rank one (a single look, e.g. an isolated persistent scatterer): every
    // |C_ik| is 1 up to the rounding of the products and reciprocal square roots
    // that normalise it (a few ulps each); G is singular, the EVD fallback
    // applies and its answer (the phases of column 0) is exact in single
    // precision.  Any other singular-looking G goes to double precision, which
    // applies the reference pivot limit.
    const bool rank_one = !is_fp64 && prm.beta == 0.f && group_min<NP, T>(mmin, gmask) >= T(1) - T(64) * Eps<T>::v;
    const T norm_g = group_max<NP, T>(live ? rs : T(0), gmask);
    T minpiv = T(1), cond = T(1), norm_gi = T(1);
    bool finite = true;
    const T pfail = T(kPivotFail), pband = is_fp64 ? T(0) : T(kPivotBand);
    if (!rank_one) {
        minpiv = gj_invert<NP, T, T, true>(g, rbuf, r, n, gmask, pfail + pband);
        T rsi = 0;
#pragma unroll
        for (int k = 0; k < NP; ++k) rsi += abs_t(g[k]);
        norm_gi = group_max<NP, T>(live ? rsi : T(0), gmask);
        cond = norm_g * norm_gi;
        finite = isfinite(cond);
    }
    // Decision: a pivot clearly below the limit fails, one clearly above
    // passes; a pivot inside the band (or a non-finite inverse without a clear
    // failure) is decided in double precision.
    const bool clear_fail = rank_one || minpiv <= pfail - pband;
    const bool ambiguous = !clear_fail && (minpiv <= pfail + pband || !finite);
    if (!is_fp64 && prm.fp64_resolve && !clear_fail && (ambiguous || cond > T(prm.cond_max))) {
        out.flag = true;
        return out;
    }
    const bool inv_failed = clear_fail || (minpiv <= pfail) || !finite;
    // G^{-1} row: kept in g, or parked in gslot (GSM) and read back by with_g.
    auto put_g = [&](const T (&src)[NP]) {
        if constexpr (GSM) {
            constexpr int E = 16 / sizeof(T);
#pragma unroll
            for (int q = 0; q < NP / E; ++q) {
                uint4 v;
                memcpy(&v, &src[q * E], 16);
                reinterpret_cast<uint4 *>(gslot)[q] = v;
            }
        }
    };
    auto with_g = [&](auto &&f) {
        if constexpr (GSM) {
            constexpr int E = 16 / sizeof(T);
            T gg[NP];
#pragma unroll
            for (int q = 0; q < NP / E; ++q) {
                const uint4 v = reinterpret_cast<const uint4 *>(gslot)[q];
                memcpy(&gg[q * E], &v, 16);
            }
            return f(gg);
        } else {
            return f(g);
        }
    };
    put_g(g);

    T mu = T(prm.mu);
    if (inv_failed) load_crow<NP, T>(a, load, r, n);  // EVD fallback: power iteration on C first

    // Start vector: phases of column 0 of C (the interferograms to entry 0).
    cpx<T> x;
    {
        const cpx<T> c0 = (live ? load(0) : mk<T>(T(0), T(0)));
        const T m2 = norm2(c0);
        x = (m2 > T(0)) ? (rsqrt_t(m2) * c0) : mk<T>(T(1), T(0));
        x = live ? (rsqrt_t(T(n)) * x) : mk<T>(T(0), T(0));
    }
    const T tol = is_fp64 ? T(1e-9) : T(prm.tol);
    cpx<T> d;
    T q;
    auto reform = [&](T m) {
        return with_g([&](const T (&gg)[NP]) { return form_shift_inverse<NP, T>(a, gg, load, m, cbuf, r, n, gmask); });
    };
    // Pass 0: EMI (shifted inverse iteration on A = G^-1 o C), or on the EVD
    // fallback power iteration on C.  Power iteration converges like
    // lambda_2 / lambda_1 = q; when that is slow its stopping rule leaves an
    // error of about tol q / (1 - q) on the unit eigenvector, which a small entry
    // turns into a phase error above the single-precision target, so pass 1
    // refines by shifted inverse iteration on -C (its smallest eigenvector is the
    // largest one of C; g = -1 makes A = g o C = -C) from a shift just below
    // -lambda_1: rho = x^H C x <= lambda_1 and lambda_1 - lambda_2 ~ (1 - q) rho;
    // a shift that is not below it fails the inertia check and is rebuilt at
    // -1.001 ||C||_inf.  One call site keeps the inlined iteration single.
    // max_iter caps the steps of both passes together: the power iteration
    // stops as soon as it is seen to be slow, and the refinement gets what it
    // left.
    bool conv = false, refined = false, evd_power = inv_failed;
    T fl_num = T(0.999), fl_den = norm_g;
    int budget = prm.max_iter;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        int used = 0;
        conv = inverse_iteration<NP, T>(a, x, d, mu, q, reform, !evd_power, cbuf, r, live, gmask, tol, budget,
                                        !evd_power, fl_num, fl_den, &used, evd_power);
        budget -= used;
        if (!(evd_power && (!conv || q > T(0.3)) && budget > 0)) break;
        const T rho = d.x;
        T cs = T(0);
#pragma unroll
        for (int k = 0; k < NP; ++k) cs += mag_t(norm2(a[k]));  // a still holds C
        const T cn = group_max<NP, T>(live ? cs : T(0), gmask);
#pragma unroll
        for (int k = 0; k < NP; ++k) g[k] = T(-1);
        put_g(g);
        mu = -(rho + T(0.1) * fmax(T(1) - q, T(0.01)) * rho);
        fl_num = -T(1.001) * cn;
        fl_den = T(1);
        evd_power = false;
        refined = true;
    }
    if (conv && (!inv_failed || refined)) {
        // Residual correction against A itself: x <- x - B^{-1} (A x - rho x).
        // Its fixed point is an exact eigenvector of A, whatever the rounding
        // of the computed B^{-1} (preconditioned inverse iteration).
        const cpx<T> ax =
            with_g([&](const T (&gg)[NP]) { return apply_A<NP, T>(gg, load, x, cbuf, r, n, gmask); });
        const T rho = group_sum<NP, T>(live ? (x.x * ax.x + x.y * ax.y) : T(0), gmask);
        const cpx<T> res = live ? (ax - rho * x) : mk<T>(T(0), T(0));
        cpx<T> corr = group_matvec<NP, T>(a, res, cbuf, r, gmask);
        cpx<T> xn = live ? (x - corr) : mk<T>(T(0), T(0));
        const T s2 = group_sum<NP, T>(norm2(xn), gmask);
        if (s2 > T(0)) x = rsqrt_t(s2) * xn;
    }
    // x^H B^{-1} x = 1 / (lambda - mu) at convergence (lambda of A; -lambda_max(C)
    // on the fallback, whose eigenvalue is not reported).
    const T theta = T(1) / ((d.x != T(0)) ? d.x : Lim<T>::tiny);
    const T lam = mu + theta;

    if (!is_fp64 && prm.fp64_resolve && !inv_failed) {
        // gap = lambda_2 - lambda_1 from q = theta / (lambda_2 - mu)
        const T gap = (q > T(0)) ? abs_t(theta) * (T(1) / q - T(1)) : abs_t(theta) * T(1e3);
        const T est = T(4) * Eps<T>::v * cond * norm_gi / fmax(gap, Lim<T>::tiny);
        if (!conv || !(est <= T(prm.err_max))) {
            out.flag = true;
            return out;
        }
    }

    // Reference (Sec. II-A): phihat_i = arg(v_i conj(v_ref)), phihat_ref = 0.
    cpx<T> vr;
    vr.x = __shfl_sync(gmask, x.x, glane0 + ref);
    vr.y = __shfl_sync(gmask, x.y, glane0 + ref);
    const cpx<T> w = x * conj(vr);
    T ph = atan2_t(w.y, w.x);
    if (r == ref || !live) ph = T(0);

    // gamma_t = |sum_{i<k} (C_ik / |C_ik|) conj(zeta_i) zeta_k| / (n(n-1)/2),
    // zeta = exp(j phihat); an exactly-zero C_ik counts as phase 0.
    const T wm2 = norm2(w);
    cpx<T> zeta = (wm2 > T(0)) ? (rsqrt_t(wm2) * w) : mk<T>(T(1), T(0));
    if (r == ref) zeta = mk<T>(T(1), T(0));
    load_crow<NP, T>(a, load, r, n);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const T m2 = norm2(a[k]);
        const cpx<T> uk = (m2 > T(0)) ? (rsqrt_t(m2) * a[k]) : mk<T>(T(1), T(0));
        a[k] = (k > r && k < n) ? uk : mk<T>(T(0), T(0));
    }
    const cpx<T> rowsum = group_matvec<NP, T>(a, zeta, cbuf, r, gmask);
    const cpx<T> term = live ? (conj(zeta) * rowsum) : mk<T>(T(0), T(0));
    const T sx = group_sum<NP, T>(term.x, gmask);
    const T sy = group_sum<NP, T>(term.y, gmask);
    const T tcoh = sqrt_t(sx * sx + sy * sy) / (T(0.5) * T(n) * T(n - 1));

    out.phase = (float)ph;
    out.tcoh = (float)tcoh;
    out.v = mk<float>((float)x.x, (float)x.y);
    out.evd = inv_failed;
    out.lam = inv_failed ? __int_as_float(0x7fc00000) : (float)lam;
    out.status = !conv ? PLK_PX_NOCONV : (inv_failed ? PLK_PX_EVD : (is_fp64 ? PLK_PX_EMI_FP64 : PLK_PX_EMI));
    return out;
}

// Double-precision re-solve, mixed: the quantities the answer depends on are
// formed in double precision -- the coherence row (from `load`), G^{-1} and
// A = G^{-1} o C, the residual A x - rho x and rho -- while the shifted
// inverse B^{-1} is formed and applied in single precision as a
// preconditioner.  The single-precision inverse iteration (with the same
// shift refinement) converges first; then x <- x - B^{-1}(A x - rho x) runs in
// double precision until the correction vanishes, so the fixed point is an
// eigenvector of the double-precision A (preconditioned inverse iteration).
// The inversion of G fails (EVD fallback) when a double-precision pivot is <=
// kPivotFail; the decision is the double-precision one, and the same
// preconditioned iteration then runs on A = -C (its smallest eigenvector is the
// largest one of C); the reference phase and gamma_t run in single precision.
template <int NP, class Loader>
__device__ PixelResult emi_solve_mixed(const Loader &load, int r, int n, int ref, const EmiParams &prm,
                                       cpx<double> *dbuf, unsigned gmask, int glane0) {
    PixelResult out;
    out.flag = false;
    const bool live = r < n;
    cpx<float> *fbuf = reinterpret_cast<cpx<float> *>(dbuf);

    cpx<double> A[NP];
    load_crow<NP, double>(A, load, r, n);
    double g[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        double m = sqrt(norm2(A[k]));
        if (prm.beta != 0.f) m = (1.0 - (double)prm.beta) * m + ((k == r) ? (double)prm.beta : 0.0);
        g[k] = m;
    }
    double grow = 0.0;  // row r of |G| summed: ||G||_inf is the group maximum
#pragma unroll
    for (int k = 0; k < NP; ++k) grow += fabs(g[k]);
    const float g_norm = (float)group_max<NP, double>(live ? grow : 0.0, gmask);
    const double minpiv =
        gj_invert<NP, double, double, true>(g, reinterpret_cast<double *>(dbuf), r, n, gmask, kPivotFail);
    double gs = 0.0;
#pragma unroll
    for (int k = 0; k < NP; ++k) gs += fabs(g[k]);
    const bool inv_failed = !(minpiv > kPivotFail) || !isfinite(group_max<NP, double>(gs, gmask));

    cpx<double> x64;
    double lam = 0.0;
    bool conv = false;
    const double tol64 = 1e-9;
    {
        // A = G^-1 o C (EMI), or -C on the EVD fallback decided here in double
        // precision (its smallest eigenvector is the largest one of C), with a
        // starting shift below lambda_min(A): mu, or -1.001 ||C||_inf.
        float mu0 = prm.mu, floor_num = 0.999f, floor_den = g_norm;
        if (inv_failed) {
            double cs = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) cs += sqrt(norm2(A[k]));
            const double cn = group_max<NP, double>(live ? cs : 0.0, gmask);
#pragma unroll
            for (int k = 0; k < NP; ++k) A[k] = mk<double>(-A[k].x, -A[k].y);
            mu0 = -1.001f * (float)cn;
            floor_num = mu0;
            floor_den = 1.f;
        } else {
#pragma unroll
            for (int k = 0; k < NP; ++k) A[k] = mk<double>(g[k] * A[k].x, g[k] * A[k].y);
        }
        cpx<float> B[NP];
        auto formB = [&](float m) {
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                B[k] = mk<float>((float)A[k].x, (float)A[k].y);
                if (k == r) B[k].x -= m;
            }
            return gj_invert<NP, float, cpx<float>, false>(B, fbuf, r, n, gmask, 0.f);
        };
        float mu = mu0;
        cpx<float> x;
        {
            const cpx<double> c0 = live ? load(0) : mk<double>(0.0, 0.0);
            const double m2 = norm2(c0);
            const cpx<double> u = (m2 > 0.0) ? (rsqrt(m2) * c0) : mk<double>(1.0, 0.0);
            x = live ? mk<float>((float)(u.x * rsqrt((double)n)), (float)(u.y * rsqrt((double)n)))
                     : mk<float>(0.f, 0.f);
        }
        cpx<float> d;
        float q;
        inverse_iteration<NP, float>(B, x, d, mu, q, formB, true, fbuf, r, live, gmask, 1e-6f, prm.max_iter, true,
                                     floor_num, floor_den);
        // Tighten the preconditioner for the double-precision phase: shift to
        // just under lambda_min (by a tenth of the gap measured through q, at
        // most half the current distance), kept only if B stays positive
        // definite.  The correction then contracts by about the new ratio
        // (lambda_min - mu)/(lambda_2 - mu) per step.
        {
            const float theta = 1.f / ((d.x != 0.f) ? d.x : 1e-30f);  // lambda_min - mu
            const float gap = (q > 0.f) ? theta * (1.f / q - 1.f) : 10.f * theta;
            const float step = fminf(0.5f * theta, 0.1f * gap);
            if (theta > 0.f && step > 0.f) {
                const float mu_new = mu + (theta - step);
                if (formB(mu_new) > 0.f) mu = mu_new;
                else formB(mu);
            }
        }
        x64 = mk<double>((double)x.x, (double)x.y);
        double rho = 0.0;
        for (int it = 0; it < 50; ++it) {
            const cpx<double> ax = group_matvec<NP, double>(A, x64, dbuf, r, gmask);
            rho = group_sum<NP, double>(live ? (x64.x * ax.x + x64.y * ax.y) : 0.0, gmask);
            const cpx<double> res = live ? (ax - rho * x64) : mk<double>(0.0, 0.0);
            const cpx<float> corr = group_matvec<NP, float>(B, mk<float>((float)res.x, (float)res.y), fbuf, r, gmask);
            const cpx<double> xn = live ? (x64 - mk<double>((double)corr.x, (double)corr.y)) : mk<double>(0.0, 0.0);
            const double s2 = group_sum<NP, double>(norm2(xn), gmask);
            const double c2 = group_sum<NP, double>(live ? (double)norm2(corr) : 0.0, gmask);
            if (s2 > 0.0) x64 = rsqrt(s2) * xn;
            if (c2 <= tol64 * tol64) {
                conv = true;
                break;
            }
        }
        lam = rho;
    }

    // Reference and gamma_t (single precision from the double iterate).
    cpx<double> vr;
    vr.x = __shfl_sync(gmask, x64.x, glane0 + ref);
    vr.y = __shfl_sync(gmask, x64.y, glane0 + ref);
    const cpx<double> w = x64 * conj(vr);
    const cpx<float> wf = mk<float>((float)w.x, (float)w.y);
    float ph = atan2f(wf.y, wf.x);
    if (r == ref || !live) ph = 0.f;
    // gamma_t in single precision (as on the single-precision path).
    const float wm2 = norm2(wf);
    cpx<float> zeta = (wm2 > 0.f) ? (rsqrtf(wm2) * wf) : mk<float>(1.f, 0.f);
    if (r == ref) zeta = mk<float>(1.f, 0.f);
    cpx<float> u[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const cpx<double> cd = (live && k < n) ? load(k) : mk<double>(0.0, 0.0);
        const cpx<float> ck = mk<float>((float)cd.x, (float)cd.y);
        const float m2 = norm2(ck);
        const cpx<float> uk = (m2 > 0.f) ? (rsqrtf(m2) * ck) : mk<float>(1.f, 0.f);
        u[k] = (k > r && k < n) ? uk : mk<float>(0.f, 0.f);
    }
    const cpx<float> rowsum = group_matvec<NP, float>(u, zeta, fbuf, r, gmask);
    const cpx<float> term = live ? (conj(zeta) * rowsum) : mk<float>(0.f, 0.f);
    const float sx = group_sum<NP, float>(term.x, gmask);
    const float sy = group_sum<NP, float>(term.y, gmask);
    out.phase = ph;
    out.tcoh = sqrtf(sx * sx + sy * sy) / (0.5f * (float)n * (float)(n - 1));
    out.lam = inv_failed ? __int_as_float(0x7fc00000) : (float)lam;
    out.status = inv_failed ? PLK_PX_EVD : (conv ? PLK_PX_EMI_FP64 : PLK_PX_NOCONV);
    return out;
}

}  // namespace plk
