/*
 * plk_oracle.c -- plain, slow, FP64 CPU oracle for the sequential phase-linking
 * hot path (Staniewicz et al., "Near-Real-Time InSAR Phase Estimation for
 * Large-Scale Surface Displacement Monitoring").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path: no headers, helpers, tables or constants.
 *
 * Every step is written the way the paper states it, one pixel at a time, in
 * double precision, with no blocking or fusion:
 *   amp_stats        Sec. III-A, eqs. (merged-mean), (merged-variance)
 *   glrt_threshold   Sec. III-A (GLRT of Parizzi et al.), exact F(2n,2n) test
 *   shp_select       Sec. III-A
 *   covariance       Sec. II-A, eq. (sample-coherence), unit-power assumption
 *   phase_link       Sec. III-B, eq. (emi-eigenvalue-problem), EVD fallback;
 *                    Sec. II-A reference phase
 *   temporal_coh     Sec. III-C, eq. (temporal-coherence)
 *   compress         Sec. II-B, compressed SLC kappa = zeta^H z
 *   amp_dispersion   Sec. III-A, D_A = sigma_A / mu_A
 *   ps_regrid        Sec. IV (PS threshold on D_A) and the Supplement's
 *                    regridding of PS and DS onto the output grid
 *
 * Three quantities decide integers (the SHP mask bits and the PS flags): the per-pixel power sums
 * the threshold comparison and the amplitude dispersion.  The paper fixes no
 * precision for them, so they
 * are taken in single precision with one fixed operation order (no fused
 * multiply-add; build with -ffp-contract=off), the precision of the GPU kernel.
 * Everything else is IEEE double.
 *
 * Complex samples are interleaved (re, im) pairs.  Stacks are date-major
 * [date][row][col].  Output pixel (i, j) of a window wy x wx with strides
 * (sy, sx) is centred on input pixel (i*sy + sy/2, j*sx + sx/2).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Sec. III-B: "at pixels where the inversion of Gamma-hat fails due to numerical
 * issues".  Read as: a Cholesky pivot of the unit-diagonal G = |C| at or below
 * this value. */
#define ORC_PIVOT_FAIL 1e-4

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* S1. Amplitude statistics (Sec. III-A).                                   */
/* For each pixel: P = sum_t |z_t|^2 and A = sum_t |z_t| over the n real    */
/* SLCs, t ascending, single precision, |z|^2 = fl(fl(x*x) + fl(y*y)).      */
/* With equal weight per image (the first option of the paper, w_g = n_g), */
/* eq. (merged-mean) applied to E[A^2] = sigma^2 + mu^2 makes the merged    */
/* second moment (sum_g P_g) / (sum_g n_g); the sums are what is carried.   */
/* If accumulate != 0 the new sums are added to the values already held:   */
/* out = fl(out + new).                                                     */
/* ------------------------------------------------------------------------ */
void orc_amp_stats(const float *slc, int n, int H, int W, float *sum_pow, float *sum_amp,
                   int accumulate)
{
    const long npix = (long)H * W;
    for (long p = 0; p < npix; ++p) {
        float P = 0.0f, A = 0.0f;
        for (int t = 0; t < n; ++t) {
            const float x = slc[2 * ((long)t * npix + p)];
            const float y = slc[2 * ((long)t * npix + p) + 1];
            const float xx = x * x;
            const float yy = y * y;
            const float q = xx + yy;
            P = P + q;
            A = A + sqrtf(q);
        }
        if (accumulate) {
            sum_pow[p] = sum_pow[p] + P;
            if (sum_amp) sum_amp[p] = sum_amp[p] + A;
        } else {
            sum_pow[p] = P;
            if (sum_amp) sum_amp[p] = A;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* GLRT threshold (Sec. III-A).  For two pixels with n i.i.d. circular      */
/* Gaussian samples each, 2P/s ~ chi^2(2n), so R = P_p / P_q ~ F(2n, 2n)    */
/* exactly under equal scale, and the GLR statistic is a monotone function  */
/* of max(R, 1/R).  The size-alpha test accepts iff max/min <= c with       */
/* c = F^{-1}_{2n,2n}(1 - alpha/2).  X = P_p/(P_p+P_q) ~ Beta(n, n); with   */
/* x* = 1/(1+c), I_{x*}(n, n) = alpha/2.  For integer n the regularised     */
/* incomplete beta is the binomial tail                                     */
/*   I_x(n, n) = sum_{k=n}^{2n-1} C(2n-1, k) x^k (1-x)^(2n-1-k).            */
/* Solved for x* by bisection on (0, 1/2].                                  */
/* ------------------------------------------------------------------------ */
static double beta_nn_cdf(double x, int n)
{
    const int m = 2 * n - 1;
    double s = 0.0;
    for (int k = n; k <= m; ++k) {
        const double lc = lgamma((double)m + 1.0) - lgamma((double)k + 1.0) -
                          lgamma((double)(m - k) + 1.0);
        s += exp(lc + k * log(x) + (m - k) * log1p(-x));
    }
    return s;
}

double orc_glrt_threshold(double alpha, int n)
{
    if (!(alpha > 0.0 && alpha < 1.0) || n < 1) return NAN;
    const double target = 0.5 * alpha;
    double lo = 0.0, hi = 0.5; /* cdf(0) = 0 < target <= cdf(1/2) = 1/2 */
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (beta_nn_cdf(mid, n) < target) lo = mid; else hi = mid;
    }
    const double x = 0.5 * (lo + hi);
    return (1.0 - x) / x;
}

/* ------------------------------------------------------------------------ */
/* S2. SHP selection (Sec. III-A).  Output pixel (i, j), centre p; for each */
/* window offset (dy, dx) with q = p + (dy, dx):                            */
/*   bit (dy+hy)*wx + (dx+hx) is set iff q lies in the image, P_p > 0,      */
/*   P_q > 0 and max(P_p, P_q) <= fl(c * min(P_p, P_q)) in single precision.*/
/* A centre with P_p <= 0 (or NaN) is no-data: mask and count are zero.     */
/* mask is [Ho][Wo][nwords] with nwords = ceil(wy*wx/64); count [Ho][Wo].   */
/* ------------------------------------------------------------------------ */
void orc_shp_select(const float *sum_pow, int H, int W, int wy, int wx, int sy, int sx,
                    float c, uint64_t *mask, uint16_t *count)
{
    const int hy = wy / 2, hx = wx / 2;
    const int Ho = H / sy, Wo = W / sx;
    const int nwords = (wy * wx + 63) / 64;
    for (int i = 0; i < Ho; ++i)
        for (int j = 0; j < Wo; ++j) {
            const long o = (long)i * Wo + j;
            uint64_t *m = mask + o * nwords;
            for (int w = 0; w < nwords; ++w) m[w] = 0;
            const int cy = i * sy + sy / 2, cx = j * sx + sx / 2;
            const float Pp = sum_pow[(long)cy * W + cx];
            int cnt = 0;
            if (Pp > 0.0f) {
                for (int dy = -hy; dy <= hy; ++dy)
                    for (int dx = -hx; dx <= hx; ++dx) {
                        const int y = cy + dy, x = cx + dx;
                        if (y < 0 || y >= H || x < 0 || x >= W) continue;
                        const float Pq = sum_pow[(long)y * W + x];
                        if (!(Pq > 0.0f)) continue;
                        const float hi = Pp > Pq ? Pp : Pq;
                        const float lo = Pp > Pq ? Pq : Pp;
                        const float lim = c * lo;
                        if (hi <= lim) {
                            const int b = (dy + hy) * wx + (dx + hx);
                            m[b / 64] |= (uint64_t)1 << (b % 64);
                            ++cnt;
                        }
                    }
            }
            count[o] = (uint16_t)cnt;
        }
}

/* ------------------------------------------------------------------------ */
/* S3. Sample coherence (Sec. II-A, eq. (sample-coherence)).                */
/* S_ik = sum_{q in Omega(p)} z_i(q) conj(z_k(q)), q in mask-bit order;     */
/* with the unit-power assumption of Sec. II-A the coherence is             */
/* C_ik = S_ik / sqrt(S_ii S_kk), C_ii = 1, and C_ik = 0 where S_ii or S_kk */
/* is zero.  A pixel with an empty neighbourhood is no-data: C = NaN.       */
/* z is complex128 [N][H][W]; C is [Ho][Wo][N(N+1)/2], upper triangle by    */
/* rows: entry (i, k), i <= k, at i*N - i*(i-1)/2 + (k - i).                */
/* ------------------------------------------------------------------------ */
static long packed_index(int N, int i, int k) { return (long)i * N - (long)i * (i - 1) / 2 + (k - i); }

void orc_covariance(const double *z, int N, int H, int W, int wy, int wx, int sy, int sx,
                    const uint64_t *mask, double *C)
{
    const int hy = wy / 2, hx = wx / 2;
    const int Ho = H / sy, Wo = W / sx;
    const int nwords = (wy * wx + 63) / 64;
    const long npix = (long)H * W;
    const long ntri = (long)N * (N + 1) / 2;
    const cplx *zc = (const cplx *)z;
#pragma omp parallel for schedule(dynamic, 16)
    for (long o = 0; o < (long)Ho * Wo; ++o) {
        const int i0 = (int)(o / Wo), j0 = (int)(o % Wo);
        const int cy = i0 * sy + sy / 2, cx = j0 * sx + sx / 2;
        const uint64_t *m = mask + o * nwords;
        cplx *Cp = (cplx *)C + o * ntri;
        cplx *S = (cplx *)calloc((size_t)N * N, sizeof(cplx));
        int L = 0;
        for (int dy = -hy; dy <= hy; ++dy)
            for (int dx = -hx; dx <= hx; ++dx) {
                const int b = (dy + hy) * wx + (dx + hx);
                if (!((m[b / 64] >> (b % 64)) & 1u)) continue;
                const long q = (long)(cy + dy) * W + (cx + dx);
                ++L;
                for (int i = 0; i < N; ++i)
                    for (int k = 0; k < N; ++k)
                        S[i * N + k] += zc[i * npix + q] * conj(zc[k * npix + q]);
            }
        for (int i = 0; i < N; ++i)
            for (int k = i; k < N; ++k) {
                cplx v;
                if (L == 0) {
                    v = NAN + NAN * I;
                } else if (i == k) {
                    v = 1.0;
                } else {
                    const double sii = creal(S[i * N + i]), skk = creal(S[k * N + k]);
                    v = (sii > 0.0 && skk > 0.0) ? S[i * N + k] / sqrt(sii * skk) : 0.0;
                }
                Cp[packed_index(N, i, k)] = v;
            }
        free(S);
    }
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigendecomposition of a real symmetric n x n matrix        */
/* (Golub & Van Loan, "Matrix Computations", Sec. 8.5, cyclic-by-row        */
/* Jacobi with the symmetric 2x2 Schur decomposition).  a is overwritten;   */
/* on return w holds the eigenvalues ascending and the columns of v the     */
/* matching orthonormal eigenvectors (v row-major, v[r*n + col]).          */
/* ------------------------------------------------------------------------ */
static void jacobi_eig(int n, double *a, double *w, double *v)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) v[r * n + c] = (r == c) ? 1.0 : 0.0;
    double frob = 0.0;
    for (int r = 0; r < n * n; ++r) frob += a[r] * a[r];
    frob = sqrt(frob);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * a[p * n + q] * a[p * n + q];
        if (sqrt(off) <= 1e-15 * frob || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[p * n + q];
                if (apq == 0.0) continue;
                const double tau = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A */
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) { /* V <- V J */
                    const double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int r = 0; r < n; ++r) w[r] = a[r * n + r];
    /* selection sort, ascending, carrying eigenvector columns */
    for (int r = 0; r < n; ++r) {
        int mi = r;
        for (int c = r + 1; c < n; ++c)
            if (w[c] < w[mi]) mi = c;
        if (mi != r) {
            const double t = w[r]; w[r] = w[mi]; w[mi] = t;
            for (int k = 0; k < n; ++k) {
                const double tv = v[k * n + r];
                v[k * n + r] = v[k * n + mi];
                v[k * n + mi] = tv;
            }
        }
    }
}

/* Eigen-decomposition of an N x N Hermitian matrix through its real        */
/* symmetric embedding [[X, -Y], [Y, X]] for M = X + jY: every eigenvalue  */
/* of M appears twice, and an eigenvector [u; v] of the embedding gives the */
/* complex eigenvector u + jv.  `which` = 0 returns the eigenvector of the  */
/* smallest eigenvalue, 1 that of the largest.  lam = that eigenvalue, gap  */
/* = distance to the next distinct eigenvalue (sorted index 2 or 2N-3).     */
static void hermitian_extreme(int N, const cplx *M, int which, cplx *vec, double *lam, double *gap)
{
    const int n = 2 * N;
    double *a = (double *)malloc(sizeof(double) * n * n);
    double *v = (double *)malloc(sizeof(double) * n * n);
    double *w = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < N; ++k) {
            const double x = creal(M[i * N + k]), y = cimag(M[i * N + k]);
            a[i * n + k] = x;
            a[i * n + (k + N)] = -y;
            a[(i + N) * n + k] = y;
            a[(i + N) * n + (k + N)] = x;
        }
    jacobi_eig(n, a, w, v);
    const int col = which ? n - 1 : 0;
    for (int i = 0; i < N; ++i) vec[i] = v[i * n + col] + I * v[(i + N) * n + col];
    *lam = w[col];
    if (N >= 2) *gap = which ? (w[n - 1] - w[n - 3]) : (w[2] - w[0]);
    else *gap = INFINITY;
    free(a);
    free(v);
    free(w);
}

/* Cholesky factorisation G = L L^T of a real symmetric matrix; returns 0   */
/* when every pivot exceeds piv_min, else 1 ("the inversion fails").        */
static int cholesky(int N, const double *G, double *L, double piv_min)
{
    memset(L, 0, sizeof(double) * N * N);
    for (int j = 0; j < N; ++j) {
        double d = G[j * N + j];
        for (int k = 0; k < j; ++k) d -= L[j * N + k] * L[j * N + k];
        if (!(d > piv_min)) return 1;
        L[j * N + j] = sqrt(d);
        for (int i = j + 1; i < N; ++i) {
            double s = G[i * N + j];
            for (int k = 0; k < j; ++k) s -= L[i * N + k] * L[j * N + k];
            L[i * N + j] = s / L[j * N + j];
        }
    }
    return 0;
}

/* G^{-1} from G = L L^T: solve L Y = I, then L^T X = Y, column by column. */
static void cholesky_inverse(int N, const double *L, double *X)
{
    double *y = (double *)malloc(sizeof(double) * N);
    for (int col = 0; col < N; ++col) {
        for (int i = 0; i < N; ++i) {
            double s = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * y[k];
            y[i] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * X[k * N + col];
            X[i * N + col] = s / L[i * N + i];
        }
    }
    free(y);
}

/* ------------------------------------------------------------------------ */
/* S6. Temporal coherence (Sec. III-C, eq. (temporal-coherence)):           */
/* gamma_t = | sum_{i<k} exp(j (phi_ik - phihat_ik)) | / (N(N-1)/2), with   */
/* phi_ik = arg C_ik (arg 0 taken as 0) and phihat_ik = phihat_i - phihat_k.*/
/* C is the full N x N matrix.                                             */
/* ------------------------------------------------------------------------ */
double orc_temporal_coherence_full(int N, const cplx *C, const double *phihat)
{
    cplx s = 0.0;
    for (int i = 0; i < N; ++i)
        for (int k = i + 1; k < N; ++k) {
            const double phi_ik = atan2(cimag(C[i * N + k]), creal(C[i * N + k]));
            s += cexp(I * (phi_ik - (phihat[i] - phihat[k])));
        }
    return cabs(s) / (0.5 * N * (N - 1));
}

/* Packed-input form of the above, for tests: C packed [N(N+1)/2]. */
double orc_temporal_coherence(int N, const double *Cpacked, const double *phihat)
{
    cplx *M = (cplx *)malloc(sizeof(cplx) * N * N);
    const cplx *Cp = (const cplx *)Cpacked;
    for (int i = 0; i < N; ++i)
        for (int k = i; k < N; ++k) {
            M[i * N + k] = Cp[packed_index(N, i, k)];
            M[k * N + i] = conj(Cp[packed_index(N, i, k)]);
        }
    const double g = orc_temporal_coherence_full(N, M, phihat);
    free(M);
    return g;
}

/* ------------------------------------------------------------------------ */
/* S4-S6. Phase linking (Sec. III-B, eq. (emi-eigenvalue-problem)).         */
/* Per pixel, from the coherence C:                                         */
/*   G = (1 - beta)|C| + beta I   (beta = 0 is the paper's plug-in |C|)     */
/*   Cholesky of G; a pivot <= 1e-4 (G has unit diagonal) means the        */
/*   inversion fails -- G is indefinite, which |C| of a highly coherent C    */
/*   often is, or too close to singular to invert reliably -- and the EVD    */
/*   fallback is used: v = eigenvector of the largest eigenvalue of C       */
/*   (status 2).  Otherwise A = G^{-1} o C (Hadamard) and v = eigenvector  */
/*   of the smallest eigenvalue of A (status 0), from a full Jacobi         */
/*   eigendecomposition (an algorithm independent of any GPU solver).       */
/*   Reference (Sec. II-A): phihat_i = arg(v_i conj(v_r)), so phihat_r = 0. */
/*   gamma_t from eq. (temporal-coherence).                                 */
/* No-data (NaN) coherence gives status 3 and NaN outputs.                  */
/* Outputs: phase [N][npx], tcoh [npx], lam [npx] (lambda_min of A, NaN on  */
/* fallback), gap [npx] (distance from the selected eigenvalue to the next  */
/* one), condG [npx] (2-norm condition number of G, optional), status.      */
/* ------------------------------------------------------------------------ */
void orc_phase_link(const double *Cpacked, int N, long npx, int ref, double beta,
                    double *phase, double *tcoh, double *lam, double *gap, double *condG,
                    uint8_t *status)
{
    const long ntri = (long)N * (N + 1) / 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (long p = 0; p < npx; ++p) {
        const cplx *Cp = (const cplx *)Cpacked + p * ntri;
        cplx *C = (cplx *)malloc(sizeof(cplx) * N * N);
        cplx *A = (cplx *)malloc(sizeof(cplx) * N * N);
        double *G = (double *)malloc(sizeof(double) * N * N);
        double *L = (double *)malloc(sizeof(double) * N * N);
        double *Gi = (double *)malloc(sizeof(double) * N * N);
        cplx *v = (cplx *)malloc(sizeof(cplx) * N);
        double *ph = (double *)malloc(sizeof(double) * N);
        int nodata = 0;
        for (int i = 0; i < N; ++i)
            for (int k = i; k < N; ++k) {
                const cplx c = Cp[packed_index(N, i, k)];
                if (isnan(creal(c)) || isnan(cimag(c))) nodata = 1;
                C[i * N + k] = c;
                C[k * N + i] = conj(c);
            }
        if (nodata) {
            for (int i = 0; i < N; ++i) phase[(long)i * npx + p] = NAN;
            tcoh[p] = NAN;
            lam[p] = NAN;
            gap[p] = NAN;
            if (condG) condG[p] = NAN;
            status[p] = 3;
        } else {
            for (int i = 0; i < N; ++i)
                for (int k = 0; k < N; ++k)
                    G[i * N + k] = (1.0 - beta) * cabs(C[i * N + k]) + (i == k ? beta : 0.0);
            if (condG) {
                double *gw = (double *)malloc(sizeof(double) * N);
                double *gv = (double *)malloc(sizeof(double) * N * N);
                double *ga = (double *)malloc(sizeof(double) * N * N);
                memcpy(ga, G, sizeof(double) * N * N);
                jacobi_eig(N, ga, gw, gv);
                condG[p] = (gw[0] > 0.0) ? gw[N - 1] / gw[0] : INFINITY;
                free(gw);
                free(gv);
                free(ga);
            }
            double l, g;
            if (cholesky(N, G, L, ORC_PIVOT_FAIL) == 0) {
                cholesky_inverse(N, L, Gi);
                for (int i = 0; i < N; ++i)
                    for (int k = 0; k < N; ++k) A[i * N + k] = Gi[i * N + k] * C[i * N + k];
                hermitian_extreme(N, A, 0, v, &l, &g);
                status[p] = 0;
                lam[p] = l;
            } else {
                hermitian_extreme(N, C, 1, v, &l, &g);
                status[p] = 2;
                lam[p] = NAN;
            }
            gap[p] = g;
            for (int i = 0; i < N; ++i) {
                const cplx w = v[i] * conj(v[ref]);
                ph[i] = atan2(cimag(w), creal(w));
                phase[(long)i * npx + p] = ph[i];
            }
            tcoh[p] = orc_temporal_coherence_full(N, C, ph);
        }
        free(C);
        free(A);
        free(G);
        free(L);
        free(Gi);
        free(v);
        free(ph);
    }
}

/* ------------------------------------------------------------------------ */
/* S7. Compressed SLC (Sec. II-B): kappa = zeta^H z = sum over the real     */
/* SLCs i in [first_real, N) of exp(-j phihat_i) z_i, a plain sum.  Each    */
/* full-resolution pixel (y, x) takes the phases of the output cell whose   */
/* decimation block contains it: (min(y/sy, Ho-1), min(x/sx, Wo-1)).        */
/* A cell without phases (no-data) gives kappa = 0.                         */
/* z complex128 [N][H][W]; phase [N][Ho][Wo]; kappa complex128 [H][W].      */
/* ------------------------------------------------------------------------ */
void orc_compress(const double *z, int N, int first_real, int H, int W, int sy, int sx,
                  const double *phase, double *kappa)
{
    const int Ho = H / sy, Wo = W / sx;
    const long npix = (long)H * W, nout = (long)Ho * Wo;
    const cplx *zc = (const cplx *)z;
    cplx *kc = (cplx *)kappa;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long q = (long)y * W + x;
            if (Ho == 0 || Wo == 0) {
                kc[q] = 0.0;
                continue;
            }
            int ci = y / sy, cj = x / sx;
            if (ci > Ho - 1) ci = Ho - 1;
            if (cj > Wo - 1) cj = Wo - 1;
            const long o = (long)ci * Wo + cj;
            cplx k = 0.0;
            int bad = 0;
            for (int i = first_real; i < N; ++i) {
                const double ph = phase[(long)i * nout + o];
                if (isnan(ph)) bad = 1;
                k += cexp(-I * ph) * zc[i * npix + q];
            }
            kc[q] = bad ? 0.0 : k;
        }
}

/* ------------------------------------------------------------------------ */
/* Amplitude dispersion (Sec. III-A): D_A = sigma_A / mu_A, the mean and     */
/* standard deviation of the pixel amplitude over the images seen so far.   */
/* With one weight per image, eqs. (merged-mean) and (merged-variance) give */
/* them from the running sums SA = sum A and SP = sum A^2 = sum |z|^2:      */
/*   mu = SA / n,  sigma^2 = SP / n - mu^2  (population variance, >= 0),    */
/* so that D_A = sqrt(n SP - SA^2) / SA.  That last form is the one taken:  */
/* single precision, each operation rounded as written, the difference     */
/* clamped at 0.  SA <= 0 (a pixel that was always zero) has no dispersion: */
/* NaN.                                                                     */
/* ------------------------------------------------------------------------ */
static float amp_dispersion_one(float sp, float sa, int n)
{
    if (!(sa > 0.0f)) return NAN;
    const float nsp = (float)n * sp;
    const float sa2 = sa * sa;
    float d = nsp - sa2;
    if (d < 0.0f) d = 0.0f;
    return sqrtf(d) / sa;
}

void orc_amp_dispersion(const float *sum_pow, const float *sum_amp, long npix, int n, float *da)
{
    for (long q = 0; q < npix; ++q) da[q] = amp_dispersion_one(sum_pow[q], sum_amp[q], n);
}

/* ------------------------------------------------------------------------ */
/* PS selection and regridding (Sec. IV: a pixel is a PS when D_A <= the    */
/* threshold, 0.2 in production, at full resolution; Supplement,            */
/* "Regridding PS and DS to 30 m resolution").  Each output cell covers the  */
/* sy x sx full-resolution pixels of its decimation block (the last cell    */
/* row/column also the rows/columns beyond the grid, as for compress):      */
/*   no PS in the block    -> the cell keeps its phase-linking phases;      */
/*   one PS                -> that PS's single-reference phases;            */
/*   several PS            -> those of the PS with the lowest D_A (the      */
/*                            first in row-major order on a tie).           */
/* The single-reference phase of date i at PS q is arg(z_i(q) conj z_r(q)),  */
/* r the mini-stack's reference entry, so it shares the DS phases' datum.   */
/* Those phases must be defined: a pixel with a zero sample at r or on a    */
/* real date is not taken.  phase [N-first_real][Ho][Wo] (double) and       */
/* status [Ho][Wo] are updated in place; PS cells get status ps_code.       */
/* ------------------------------------------------------------------------ */
static int ps_phases_defined(const cplx *zc, int N, int first_real, long npix, int ref, long q)
{
    if (zc[(long)ref * npix + q] == 0.0) return 0;
    for (int i = first_real; i < N; ++i)
        if (zc[(long)i * npix + q] == 0.0) return 0;
    return 1;
}

void orc_ps_regrid(const double *z, int N, int first_real, int H, int W, int sy, int sx,
                   const float *sum_pow, const float *sum_amp, int n, int ref, float da_max,
                   double *phase, uint8_t *status, int ps_code)
{
    const int Ho = H / sy, Wo = W / sx;
    const long npix = (long)H * W, nout = (long)Ho * Wo;
    const cplx *zc = (const cplx *)z;
    for (int ci = 0; ci < Ho; ++ci)
        for (int cj = 0; cj < Wo; ++cj) {
            const int y1 = (ci == Ho - 1) ? H : (ci + 1) * sy;
            const int x1 = (cj == Wo - 1) ? W : (cj + 1) * sx;
            long best_q = -1;
            float best = 0.0f;
            for (int y = ci * sy; y < y1; ++y)
                for (int x = cj * sx; x < x1; ++x) {
                    const long q = (long)y * W + x;
                    const float da = amp_dispersion_one(sum_pow[q], sum_amp[q], n);
                    if (isnan(da) || !(da <= da_max)) continue;       /* not a PS */
                    if (!ps_phases_defined(zc, N, first_real, npix, ref, q)) continue;
                    if (best_q < 0 || da < best) {
                        best_q = q;
                        best = da;
                    }
                }
            if (best_q < 0) continue;
            const long o = (long)ci * Wo + cj;
            const cplx r = zc[(long)ref * npix + best_q];
            for (int i = first_real; i < N; ++i)
                phase[(long)(i - first_real) * nout + o] = carg(zc[(long)i * npix + best_q] * conj(r));
            status[o] = (uint8_t)ps_code;
        }
}

/* ------------------------------------------------------------------------ */
/* Compressed SLC at the PS pixels (Sec. II-B, kappa = zeta^H z, with the   */
/* PS processed at full resolution, Sec. IV): a PS pixel (same test as in   */
/* orc_ps_regrid, every PS of a block, not only the selected one) is        */
/* compressed on its own single-reference phases theta_i = arg(z_i conj     */
/* z_ref), re-referenced to date shift (theta_i - theta_shift) when         */
/* shift >= 0:  kappa(q) = sum_{i >= first_real} exp(-j theta_i) z_i(q).    */
/* kappa [H][W] is overwritten at those pixels only.                         */
/* ------------------------------------------------------------------------ */
void orc_ps_compress(const double *z, int N, int first_real, int H, int W, const float *sum_pow,
                     const float *sum_amp, int n, int ref, float da_max, int shift, double *kappa)
{
    const long npix = (long)H * W;
    const cplx *zc = (const cplx *)z;
    cplx *kc = (cplx *)kappa;
    for (long q = 0; q < npix; ++q) {
        const float da = amp_dispersion_one(sum_pow[q], sum_amp[q], n);
        if (isnan(da) || !(da <= da_max)) continue;
        if (!ps_phases_defined(zc, N, first_real, npix, ref, q)) continue;
        const cplx r = zc[(long)ref * npix + q];
        const double th_s = shift >= 0 ? carg(zc[(long)shift * npix + q] * conj(r)) : 0.0;
        cplx k = 0.0;
        for (int i = first_real; i < N; ++i) {
            const double th = carg(zc[(long)i * npix + q] * conj(r)) - th_s;
            k += cexp(-I * th) * zc[(long)i * npix + q];
        }
        kc[q] = k;
    }
}
