/*
 * plk.h -- C ABI of libplk, the GB300 (sm_103a) implementation of the
 * data-parallel hot path of sequential InSAR phase linking (Staniewicz et al.,
 * "Near-Real-Time InSAR Phase Estimation for Large-Scale Surface Displacement
 * Monitoring"): SHP selection on amplitude, SHP-windowed coherence, EMI phase
 * linking, temporal coherence and compressed-SLC formation under the
 * always-first mini-stack reference scheme.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller (for example
 *    torch tensors), unless a parameter says "host".  The library never frees
 *    them and never keeps them past the call.
 *  - Complex samples are plk_c64 (interleaved float re, im; 8-byte aligned).
 *  - Stacks are date-major and row-major: [N][H][W].  Per-output-pixel arrays
 *    are [Ho][Wo] (or [N][Ho][Wo] for phases), with, for a window wy x wx and
 *    strides (sy, sx), Ho = H / sy and Wo = W / sx (integer division), and
 *    output pixel (i, j) centred on input pixel (i*sy + sy/2, j*sx + sx/2),
 *    the centre of its sy x sx decimation block (Sec. IV; Supplement S1).
 *    A window written "X x Y" in the paper has wx = X columns, wy = Y rows.
 *  - Calls are asynchronous on the context's CUDA stream.  Arguments are
 *    checked on the host before anything is launched; a bad argument returns
 *    PLK_EINVAL and launches nothing.  A launch or runtime error returns
 *    PLK_ECUDA.  plk_last_error() gives a one-line description.
 *  - Numerical outcomes of single pixels (no data, EVD fallback, ...) are
 *    data in the status array, not errors.
 *  - N (entries of one mini-stack, compressed plus real) is 2..PLK_MAX_N.
 *    Windows are odd, wy*wx <= PLK_MAX_WINDOW.
 */
#ifndef PLK_H_
#define PLK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLK_MAX_N 32
#define PLK_MAX_WINDOW 1024

typedef enum plk_status {
    PLK_OK = 0,
    PLK_EINVAL = 1,       /* bad argument; nothing was launched */
    PLK_ENOMEM = 2,       /* a library-owned allocation failed */
    PLK_ECUDA = 3,        /* CUDA launch/runtime error */
    PLK_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
    PLK_EUNSUPPORTED = 5  /* valid request this build does not provide */
} plk_status;

/* Per-pixel outcome codes written to status arrays. */
enum {
    PLK_PX_EMI = 0,       /* EMI solution, single precision */
    PLK_PX_EMI_FP64 = 1,  /* EMI solution re-solved in double precision */
    PLK_PX_EVD = 2,       /* inversion of |C| failed: EVD fallback (Sec. III-B) */
    PLK_PX_NODATA = 3,    /* zero-power centre / empty neighbourhood: NaN outputs */
    PLK_PX_NOCONV = 4,    /* inverse iteration (EMI or EVD fallback) hit max_iter;
                             last iterate kept */
    PLK_PX_PS = 5         /* output cell takes the phase of a persistent scatterer
                             (plk_ps_regrid, Supplement "Regridding PS and DS") */
};

typedef struct plk_c64 { float re, im; } plk_c64;

/* SHP search window (odd wy, wx) and output strides (sy, sx >= 1). */
typedef struct plk_window { int32_t wy, wx, sy, sx; } plk_window;

typedef struct plk_params {
    double alpha;      /* GLRT size (Sec. III-A), 0 < alpha < 1; default 1e-3 */
    float beta;        /* |C| regularisation G = (1-beta)|C| + beta I, 0 <= beta < 1;
                          default 0, the paper's plug-in |C| (Sec. III-B) */
    float mu;          /* starting inverse-iteration shift (Sec. III-B); default
                          0.99.  A shift at or above lambda_min (its B is not
                          positive definite) is replaced by 0.999/||G||_inf, a
                          lower bound, and moved up by the reshifts */
    float tol;         /* stop when the unit iterate moves less than tol (2-norm,
                          after removing a common phase); default 1e-6 */
    int32_t max_iter;  /* inverse-iteration cap, all shifts together (on the EVD
                          fallback, the power iteration and its refinement
                          together); default 100 */
    float cond_max;    /* pixels whose 1-norm condition number of G exceeds
                          cond_max, or whose single-precision inversion of G meets
                          a pivot within 2e-5 of the 1e-4 failure limit, are
                          re-solved in double precision; default 1e4 */
    int32_t fp64_resolve; /* 1 (default): re-solve flagged pixels in FP64; 0: keep
                             the single-precision result */
    float err_max;     /* pixels whose first-order single-precision error bound
                          (condition of G times |G^-1| times eps over the
                          eigengap seen by the iteration) exceeds err_max are
                          re-solved in double precision; default 0.1 (the bound
                          is loose: measured errors sit 1e3-1e4 below it) */
    int32_t cov_precision; /* coherence arithmetic (S3): PLK_COV_FP32 (default),
                              PLK_COV_BF16 (samples rounded to bfloat16, sums in
                              single precision on the tensor cores; N <= 32) or
                              PLK_COV_FP16 (the same with half-precision samples,
                              scaled by a power of two per tile; N <= 32) */
    int32_t ref_scheme;    /* mini-stack reference scheme of plk_ministack_step:
                              PLK_REF_FIRST (default) or PLK_REF_LAST_REAL */
    float ps_da_max;       /* plk_ministack_step: when > 0, output cells whose
                              decimation block holds a pixel with amplitude
                              dispersion D_A <= ps_da_max take that persistent
                              scatterer's phase (plk_ps_regrid), and every PS
                              pixel is compressed on its own phases
                              arg(z_i conj z_ref), so that later mini-stacks keep
                              its datum; default 0 (off); the paper's production
                              value is 0.2 */
    float decay;           /* plk_ministack_step: weighting of the merged
                              amplitude statistics (Sec. III-A, the exponential
                              decay option beside equal weights per image):
                              image t of the T merged so far weighs
                              decay^(T-1-t), the newest 1.  0 < decay <= 1;
                              default 1 (equal weights, the sums of
                              plk_amp_stats).  Below 1, S1 keeps decayed sums
                              (each image's power times its weight, in single
                              precision, images in order; the running sums
                              scaled by decay^M before a group of M is added)
                              and the GLRT uses nu = W1^2 / W2 effective looks
                              (W1, W2: sums of the weights and of their
                              squares) through plk_glrt_threshold_looks.  Not
                              with ps_da_max > 0 (EUNSUPPORTED) */
} plk_params;

/* Mini-stack reference schemes (plk_params.ref_scheme).  Both link each
 * mini-stack with the newest compressed SLC (or the first real SLC when there
 * is none) as reference.  PLK_REF_FIRST (Sec. II-B, Fig. 1): the new
 * compressed SLC is formed on the linked phases as they are, so every one
 * carries the phase of the archive's first date and all outputs are relative
 * to it.  PLK_REF_LAST_REAL (Sec. IV; Supplement, "Compressed SLC strategy
 * for separate batched processing"): the new compressed SLC is formed on the
 * phases re-referenced to the mini-stack's last real SLC, so it carries that
 * date's phase and the next mini-stack's outputs are short-baseline
 * interferograms relative to it. */
#define PLK_REF_FIRST 0
#define PLK_REF_LAST_REAL 1

/* Coherence precision modes (plk_params.cov_precision, plk_estimate_covariance). */
#define PLK_COV_FP32 0
#define PLK_COV_BF16 1
#define PLK_COV_FP16 2

typedef struct plk_ctx plk_ctx;
typedef struct plk_state plk_state;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out is owned by the
 * caller and released with plk_destroy; it holds an 8-byte device counter
 * (allocated here, the only allocation of a context).  Errors: EINVAL (null out, bad
 * device), ENOMEM, ECUDA. */
plk_status plk_create(plk_ctx **out, int device, void *cuda_stream);
plk_status plk_destroy(plk_ctx *ctx);
/* Switch the stream used by later calls. */
plk_status plk_set_stream(plk_ctx *ctx, void *cuda_stream);
/* Wait for the work issued on ctx's stream.  Returns PLK_ETIMEOUT if a
 * bounded device-side wait (a kernel waiting for its staged tile data) gave up
 * since the last plk_sync -- that launch's outputs are then incomplete --
 * else PLK_ECUDA on an asynchronous CUDA error, else PLK_OK. */
plk_status plk_sync(plk_ctx *ctx);
/* Failure-detection self-test (not part of the method): launches one warp that
 * waits on a device barrier nothing will complete.  Its bounded wait gives up
 * after about a second, so the next plk_sync returns PLK_ETIMEOUT and the
 * context stays usable.  Faults nothing and hangs nothing. */
plk_status plk_selftest_bounded_wait(plk_ctx *ctx);
/* Text of the last error on this context (static storage owned by ctx). */
const char *plk_last_error(const plk_ctx *ctx);
/* Fill *p with the defaults listed in plk_params. */
plk_status plk_default_params(plk_params *p);
/* Output grid of a window: *Ho = H / sy, *Wo = W / sx (host). */
plk_status plk_output_shape(int H, int W, plk_window win, int *Ho, int *Wo);
/* Mask words per output pixel: ceil(wy*wx / 64) (host). */
int plk_mask_words(plk_window win);

/* Per-kernel timing (not part of the method).  While enabled, every kernel
 * launch of a call is bracketed by CUDA events recorded on ctx's stream (up to
 * 4096 launches between collections; enabling allocates the events).
 * plk_profile_collect synchronizes the stream and aggregates the recorded
 * launches by kernel stage name ("amp_stats", "shp_select", "covariance",
 * "phase_link_fp32", "phase_link_fp64", "compress"); plk_profile_get returns
 * stage i's name (static string), total milliseconds and launch count. */
plk_status plk_profile_enable(plk_ctx *ctx, int enable);
plk_status plk_profile_collect(plk_ctx *ctx, int *n_kernels);
plk_status plk_profile_get(const plk_ctx *ctx, int i, const char **name, double *total_ms, int *launches);

/* GLRT threshold (Sec. III-A), host only.  For n_eff samples per pixel the
 * power ratio of two homogeneous pixels is F(2n, 2n) distributed, and the
 * size-alpha GLRT accepts iff max/min <= c = F^{-1}_{2n,2n}(1 - alpha/2).
 * Writes c to *c (host pointer).  EINVAL if alpha not in (0,1) or n_eff < 1. */
plk_status plk_glrt_threshold(double alpha, int n_eff, double *c);
/* The same threshold for a real number of looks nu >= 1 (Sec. III-A with
 * exponentially decaying image weights, nu = W1^2 / W2): the ratio of two
 * weighted power sums is taken as F(2 nu, 2 nu) distributed.  Equals
 * plk_glrt_threshold at integer nu.  EINVAL if alpha not in (0,1) or nu < 1. */
plk_status plk_glrt_threshold_looks(double alpha, double nu, double *c);

/* ---------------------------------------------------------- hot-path calls */

/* S1. Amplitude statistics (Sec. III-A, eqs. (merged-mean), (merged-variance)
 * with equal weight per image).  For each pixel of slc [n][H][W]:
 *   P = sum_t fl(fl(re^2) + fl(im^2)),  A = sum_t sqrt(...),  t ascending,
 * single precision, no fused multiply-add (the sums decide mask bits).
 * accumulate = 0: sum_pow = P (and sum_amp = A); accumulate = 1: sum_pow +=
 * P (one float add), which merges a new group into the running statistics.
 * sum_pow [H][W] float is required; sum_amp may be NULL.  n >= 1.
 * The sums are float, not double: the GLRT decision is taken in single
 * precision on both sides of the parity test, in a fixed order of operations,
 * so masks match bit for bit (the paper fixes no precision for it). */
plk_status plk_amp_stats(plk_ctx *ctx, const plk_c64 *slc, int n, int H, int W,
                         float *sum_pow, float *sum_amp, int accumulate);

/* S2. SHP selection by GLRT (Sec. III-A).  sum_pow [H][W] holds the power
 * sums over n_eff real images.  For output pixel p (centre as above) and
 * window offset (dy, dx), bit (dy+hy)*wx + (dx+hx) of mask[p] is set iff the
 * neighbour q is inside the image, P_p > 0, P_q > 0 and
 *   max(P_p, P_q) <= fl(c * min(P_p, P_q)),  c = (float) plk_glrt_threshold.
 * mask is [Ho][Wo][plk_mask_words(win)] uint64; count [Ho][Wo] uint16 gets the
 * number of set bits (the paper's shp_counts layer; 0 marks no-data).
 * sum_pow is float, as plk_amp_stats writes it (single-precision decision). */
plk_status plk_shp_select(plk_ctx *ctx, const float *sum_pow, int n_eff, int H, int W,
                          plk_window win, double alpha, uint64_t *mask, uint16_t *count);

/* S3. Sample coherence (Sec. II-A, eq. (sample-coherence)).  For each output
 * pixel, S_ik = sum over the set mask bits q of z_i(q) conj(z_k(q)), and
 * C_ik = S_ik / sqrt(S_ii S_kk) (unit-power assumption of Sec. II-A), C_ii = 1,
 * C_ik = 0 where S_ii or S_kk is 0; an empty mask gives NaN entries.
 * slc [N][H][W]; mask as written by plk_shp_select for the same window;
 * C_packed [Ho][Wo][N(N+1)/2], upper triangle by rows: entry (i, k), i <= k,
 * at i*N - i*(i-1)/2 + (k - i).  precision PLK_COV_FP32: single-precision
 * products and sums; PLK_COV_BF16: the samples are rounded to bfloat16 (round
 * to nearest even) and the products summed in single precision on the tensor
 * cores, N <= 32 (EUNSUPPORTED beyond); PLK_COV_FP16: the same with the
 * samples of each output tile's region scaled by one power of two (its largest
 * component into [2^14, 2^15), cancelled exactly by the normalisation) and
 * rounded to half precision (round to nearest even), N <= 32. */
plk_status plk_estimate_covariance(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W,
                                   plk_window win, const uint64_t *mask, int precision,
                                   plk_c64 *C_packed);

/* S4-S6. EMI phase linking (Sec. III-B, eq. (emi-eigenvalue-problem)) with the
 * reference of Sec. II-A and gamma_t of Sec. III-C, eq. (temporal-coherence).
 * For each of npx packed coherences C_packed [npx][N(N+1)/2]:
 *   G = (1-beta)|C| + beta I; v = eigenvector of the smallest eigenvalue of
 *   G^{-1} o C by inverse iteration with shift mu; EVD fallback (largest
 *   eigenvector of C) where the inversion of G fails;
 *   phase[i][p] = arg(v_i conj(v_ref)) in (-pi, pi], phase[ref][p] = 0;
 *   tcoh[p] = gamma_t over all N entries; lambda_min[p] = the eigenvalue
 *   (NaN on EVD fallback); status[p] as PLK_PX_*.
 * phase [N][npx] float; tcoh, lambda_min [npx] float (either may be NULL);
 * status [npx] uint8 (required).  0 <= ref_idx < N.  params NULL = defaults. */
plk_status plk_phase_link(plk_ctx *ctx, const plk_c64 *C_packed, int N, int64_t npx,
                          int ref_idx, const plk_params *params, float *phase, float *tcoh,
                          float *lambda_min, uint8_t *status);

/* S7. Compressed SLC (Sec. II-B): kappa(y, x) = sum over the real entries
 * i in [first_real, N) of exp(-j phase_i(cell)) z_i(y, x), a plain sum, where
 * cell = (min(y/sy, Ho-1), min(x/sx, Wo-1)) is the output pixel whose
 * decimation block holds (y, x).  A cell with NaN phases gives kappa = 0.
 * slc [N][H][W]; phase [N][Ho][Wo] (only rows >= first_real are read);
 * kappa [H][W].  0 <= first_real < N. */
plk_status plk_compress(plk_ctx *ctx, const plk_c64 *slc, int N, int first_real, int H, int W,
                        plk_window win, const float *phase, plk_c64 *kappa);

/* ------------------------------------------------- sequential state (S8) */

/* State of one sequential chain (Sec. II-B): the ring of the K_max most recent
 * compressed SLCs, the merged power/amplitude sums and the image count.
 * Allocates every buffer a step needs for images of H x W, window win and at
 * most M_max new SLCs per step (K_max + M_max <= PLK_MAX_N), so that
 * plk_ministack_step allocates nothing.  Owned by the caller; release with
 * plk_state_destroy.  Errors: EINVAL, ENOMEM. */
plk_status plk_state_create(plk_ctx *ctx, int H, int W, plk_window win, int K_max, int M_max,
                            plk_state **out);
plk_status plk_state_destroy(plk_state *st);
/* Start a new chain on the same buffers: the next step is a first step (its
 * statistics overwrite the sums; no compressed SLC is used).  Host only. */
plk_status plk_state_reset(plk_state *st);
/* Host-side counters: compressed SLCs held, real images merged, steps run. */
plk_status plk_state_info(const plk_state *st, int *K_used, int *n_eff, int *steps);
/* Sums of the image weights merged so far and of their squares (W1, W2;
 * both n_eff with equal weights); nu = W1^2 / W2 effective looks. */
plk_status plk_state_weights(const plk_state *st, double *W1, double *W2);
/* Device pointer to compressed SLC i of the ring (0 = oldest), [H][W]. */
plk_status plk_state_kappa(const plk_state *st, int i, const plk_c64 **kappa);
/* Device pointers to the merged sums [H][W] (sum_amp may be NULL). */
plk_status plk_state_sums(const plk_state *st, const float **sum_pow, const float **sum_amp);
/* Checkpoint: write/read the ring, sums and counters to/from a file (host
 * path).  load creates a new state (as plk_state_create) on ctx's device. */
plk_status plk_state_save(plk_ctx *ctx, const plk_state *st, const char *path);
plk_status plk_state_load(plk_ctx *ctx, const char *path, int M_max, plk_state **out);

/* S1-S8. One step of the always-first mini-stack scheme (Sec. II-B items
 * 1-3; NRT workflow steps 1-4 of Sec. III-G): merge the statistics of the M
 * new SLCs new_slc [M][H][W] into st; GLRT SHP selection with n_eff = all
 * real images so far; mini-stack = [ring oldest..newest, new SLCs]; coherence;
 * EMI with reference = the newest compressed SLC (or the first new SLC on the
 * first step); gamma_t; compress the new SLCs into a new kappa and push it
 * (dropping the oldest beyond K_max).  Outputs for the real dates only:
 * phase [M][Ho][Wo] relative to the first date of the archive (PLK_REF_FIRST)
 * or to the previous mini-stack's last real date (PLK_REF_LAST_REAL; the
 * first date on the first step), tcoh [Ho][Wo],
 * status [Ho][Wo]; shp_count [Ho][Wo] may be NULL.  With params->ps_da_max > 0
 * the output cells holding a persistent scatterer take its phases (status
 * PLK_PX_PS, tcoh unchanged; plk_ps_regrid) and each PS pixel's kappa is formed
 * on its own phases.  1 <= M <= M_max and M + (compressed SLCs held) >= 2.
 * params NULL = defaults. */
plk_status plk_ministack_step(plk_ctx *ctx, plk_state *st, const plk_c64 *new_slc, int M,
                              const plk_params *params, float *phase, float *tcoh,
                              uint8_t *status, uint16_t *shp_count);
/* S1-S8 from host memory: plk_ministack_step with the new SLCs read from host
 * memory new_slc [M][H][W] and the outputs phase [M][Ho][Wo], tcoh and status
 * [Ho][Wo] (shp_count may be NULL) written to host memory.  Asynchronous: it
 * returns once the work is enqueued; the host buffers must stay untouched
 * until plk_sync(ctx).  The SLCs go to one of two device staging buffers on a
 * copy stream of the library's own, so a call's copy overlaps the previous
 * call's compute (with pinned host memory; pageable memory works but copies
 * synchronously).  The staging buffers come from plk_state_enable_host_io,
 * which must have been called on st (EINVAL otherwise); the step itself
 * allocates nothing.  Errors: EINVAL, ECUDA, and those of plk_ministack_step.
 * Not part of the paper's method: a transfer schedule around it. */
/* Set-up for plk_ministack_step_host: allocates st's two device staging
 * buffers (M_max planes of H x W each), the device outputs, a copy stream and
 * its events; plk_state_destroy releases them.  A second call does nothing.
 * Errors: EINVAL, ENOMEM (nothing is kept). */
plk_status plk_state_enable_host_io(plk_ctx *ctx, plk_state *st);
/* Device allocations (successful cudaMalloc calls) the library has made in
 * this process: contexts, states, host-I/O staging, batches.  A diagnostic for
 * callers that must not allocate after set-up; no step or hot-path call adds
 * to it. */
int64_t plk_device_allocations(void);
plk_status plk_ministack_step_host(plk_ctx *ctx, plk_state *st, const plk_c64 *new_slc, int M,
                                   const plk_params *params, float *phase, float *tcoh, uint8_t *status,
                                   uint16_t *shp_count);
/* Set-up for plk_ministack_step_host_ci16: plk_state_enable_host_io's
 * buffers plus two device staging buffers of M_max planes of H x W complex
 * 16-bit samples.  A second call does nothing.  Errors: EINVAL, ENOMEM
 * (nothing is kept). */
plk_status plk_state_enable_host_io_ci16(plk_ctx *ctx, plk_state *st);
/* plk_ministack_step_host with the new SLCs as complex 16-bit integers:
 * new_slc [M][H][W][2] int16 (re, im interleaved, 4-byte aligned; the sample
 * format Sentinel-1 SLC products store), half the bytes of complex64 over the
 * host link.  On the device each sample is widened exactly to complex64 (every
 * int16 is a float: no scale), so the results equal those of
 * plk_ministack_step on the widened samples.  The samples go to one of two
 * int16 staging buffers on the library's copy stream; the widening runs on
 * ctx's stream before the step, and frees the buffer for the next call's copy.
 * Needs plk_state_enable_host_io_ci16 on st (EINVAL otherwise).  Asynchronous
 * as plk_ministack_step_host.  Errors: EINVAL, ECUDA, and those of
 * plk_ministack_step.  Not part of the paper's method: an input format. */
plk_status plk_ministack_step_host_ci16(plk_ctx *ctx, plk_state *st, const int16_t *new_slc, int M,
                                        const plk_params *params, float *phase, float *tcoh, uint8_t *status,
                                        uint16_t *shp_count);


/* ------------------------------------------ persistent scatterers */

/* PS selection and regridding (Sec. III-A, eq. (amplitude dispersion); Sec. IV;
 * Supplement "Regridding PS and DS to 30 m resolution").  Per full-resolution
 * pixel, D_A = sigma_A / mu_A from the merged sums, with mu = sum_amp / n_eff
 * and the population deviation sigma, taken as
 * D_A = sqrt(max(n_eff * sum_pow - sum_amp^2, 0)) / sum_amp in single
 * precision in this order with correctly rounded operations and no fused
 * multiply-add; a pixel with sum_amp > 0,
 * D_A <= da_max and nonzero samples at ref_idx and on every real date (so
 * that its phases are defined) is a PS.  Per output cell (its sy x sx decimation block; the
 * last row/column of cells also takes the rows/columns beyond the grid): with
 * no PS the phases are left as they are (the DS phase-linking result); else
 * the PS with the lowest D_A (the first in row-major order on a tie) gives
 * phase[j][cell] = arg(z_{first_real+j}(q) conj(z_ref(q))) for every real date
 * j, and status[cell] = PLK_PX_PS.  slc [N][H][W] (the mini-stack, reference
 * entry ref_idx); sum_pow, sum_amp [H][W]; phase [N-first_real][Ho][Wo] and
 * status [Ho][Wo] are updated in place.  Errors: EINVAL, ECUDA. */
plk_status plk_ps_regrid(plk_ctx *ctx, const plk_c64 *slc, int N, int first_real, int H, int W, plk_window win,
                         const float *sum_pow, const float *sum_amp, int n_eff, int ref_idx, float da_max,
                         float *phase, uint8_t *status);

/* Phase cosine similarity gamma_s (Sec. III-C, eq. (phase-cosine-sim)).  For
 * each output pixel p of the linked phases phase [M][Ho][Wo] (float, e.g. the
 * real dates of a step's output) and each neighbour x of the disk
 * dy^2 + dx^2 <= radius^2 (p itself excluded; neighbours outside the grid or
 * with a non-finite phase left out):
 *   s(p, x) = (1/N_ifg) sum cos((phi_b - phi_a)(p) - (phi_b - phi_a)(x))
 * over the nearest-3 network, the pairs (a, b) with 1 <= b - a <= 3
 * (N_ifg = 3M - 6 for M >= 3); gamma_s[p] = the median of s(p, x) over x (the
 * mean of the two middle values for an even count), NaN where p has a
 * non-finite phase or no neighbour is left.  gamma_s [Ho][Wo] float.  The
 * paper's window is ~200 m (radius 7 at a 30 m posting).  2 <= M <= 32,
 * 1 <= radius <= 32.  Errors: EINVAL; EUNSUPPORTED where the disk holds more
 * than 512 neighbours (radius > 12) or the window and M exceed a CTA's shared
 * memory; ECUDA. */
plk_status plk_phase_similarity(plk_ctx *ctx, const float *phase, int M, int Ho, int Wo, int radius,
                                float *gamma_s);

/* L1 time-series network inversion by ADMM (Sec. III-E, eq. (l1-min);
 * Appendix).  Per pixel p, with b = unw[k][p] the unwrapped phase of
 * interferogram k = (pairs[2k], pairs[2k+1]) = (a, b), a < b, and x the
 * phase series of dates 1..n_dates-1 relative to date 0, minimise
 * ||A x - b||_1 (A: -1 at date a, +1 at date b) by the ADMM iteration
 *   x = (A^T A)^{-1} A^T (b + z - u),  z = S_{1/rho}(A x - b + u),
 *   u = u + A x - b - z,
 * from z = u = 0, exactly `iters` iterations, in single precision (the
 * Cholesky factor of A^T A, shared by all pixels, in double on the host).
 * Networks: any set of distinct pairs with b - a <= 3 (the nearest-3 network
 * of Sec. III-D and its subsets) that determines every date; n_dates <= 17.
 * unw [n_ifg][npx] float (device); pairs [n_ifg][2] int32 (host); x
 * [n_dates-1][npx] float; residual [n_ifg][npx] float = b - A x (may be NULL:
 * residuals far from 2 pi k mark unwrapping errors, Sec. III-E).  rho > 0,
 * 1 <= iters <= 100000.  Errors: EINVAL (bad pair, repeated pair, a network
 * that leaves a date undetermined); EUNSUPPORTED (b - a > 3, n_dates > 17);
 * ECUDA. */
plk_status plk_invert_l1(plk_ctx *ctx, const float *unw, int n_dates, const int32_t *pairs, int n_ifg, int64_t npx,
                         float rho, int iters, float *x, float *residual);

/* ----------------------------------------------------------- adjoint */

/* Scratch bytes plk_phase_link_backward needs for this stack and window. */
plk_status plk_backward_workspace_size(int N, int H, int W, plk_window win, size_t *bytes);
/* Adjoint of S3-S5 (coherence, Sec. II-A; EMI eigenvector, Sec. III-B;
 * referenced phase, Sec. II-A) with the SHP masks frozen: for
 * L = sum_{i,p} dphase[i][p] * phase[i][p], where phase is what
 * plk_estimate_covariance + plk_phase_link (single-precision solve, same mask,
 * ref_idx and params) produce, writes dslc [N][H][W] with
 * dL = Re sum conj(dslc) dz, i.e. dslc = dL/dRe z + j dL/dIm z.
 * The eigenvector derivative is the first-order perturbation of a simple
 * eigenvalue (it grows as 1 / eigengap); the coherence is recomputed, not
 * stored.  slc [N][H][W]; mask as from plk_shp_select; dphase [N][Ho][Wo];
 * workspace: device memory of plk_backward_workspace_size bytes, owned by
 * the caller (nothing is allocated).  Pixels without data contribute nothing.
 * N <= 32.  Errors: EINVAL (bad argument, small workspace), ECUDA.  The paper
 * states no adjoint. */
plk_status plk_phase_link_backward(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                   const uint64_t *mask, int ref_idx, const plk_params *params,
                                   const float *dphase, void *workspace, size_t workspace_bytes,
                                   plk_c64 *dslc);

/* Gradient of L = sum(dphase * phase) with respect to real per-sample window
 * weights, the SHP mask read as weights w_b in the sample covariance
 * S = sum_b w_b z(q_b) z(q_b)^H (Sec. II-A, eq. (sample-coherence) with a
 * weighted sum), evaluated at w = mask: dL/dw_b = (1/2) z(q_b)^H H_p z(q_b),
 * H_p the adjoint's matrix of pixel p (see plk_phase_link_backward).  Samples
 * outside the mask get the derivative of adding them with a small weight;
 * samples outside the image and pixels without data get 0.  Scaling every
 * weight of a pixel leaves its coherence unchanged, so the sum over its
 * masked samples is 0.  dweight [Ho][Wo][wy*wx] float, b = (dy + wy/2) * wx +
 * (dx + wx/2) as in the mask bits.  Workspace as plk_backward_workspace_size.
 * Errors: EINVAL, EUNSUPPORTED, ECUDA. */
plk_status plk_shp_weight_gradient(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                   const uint64_t *mask, int ref_idx, const plk_params *params,
                                   const float *dphase, void *workspace, size_t workspace_bytes, float *dweight);

/* Phase uncertainty through the adjoint: the first-order standard deviation
 * of every linked phase when white circular Gaussian noise of variance sigma2
 * (E|n|^2 = sigma2) is added to every SLC sample, SHP masks frozen.  For
 * pixel p and date i, with g(q) = H z(q) the adjoint's gradient of phihat_i(p)
 * over the pixel's masked window, Var phihat_i = (sigma2 / 2) sum_q |g(q)|^2 =
 * (sigma2 / 2) tr(H^H H S), S = sum_q m(q) z(q) z(q)^H (the pixel's
 * unnormalised sample covariance); one adjoint solve per date, no window
 * scatter.  phase_std [N][Ho][Wo] float: 0 at ref_idx, NaN without data.
 * Workspace as plk_backward_workspace_size.  Not in the paper (it applies the
 * adjoint to uncertainty propagation).  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
plk_status plk_phase_uncertainty(plk_ctx *ctx, const plk_c64 *slc, int N, int H, int W, plk_window win,
                                 const uint64_t *mask, int ref_idx, const plk_params *params, float sigma2,
                                 void *workspace, size_t workspace_bytes, float *phase_std);

/* ------------------------------------------------ batches of stacks */

/* One independent stack of a batch: its SLCs and where its outputs go (all
 * device pointers, owned by the caller, fixed for the batch's life). */
typedef struct plk_stack_desc {
    const plk_c64 *slc;  /* [N][H][W] */
    int32_t N, H, W;     /* 2 <= N <= PLK_MAX_N; H, W >= 1 */
    int32_t ref_idx;     /* reference date of the linked phases, 0 <= ref_idx < N */
    float *phase;        /* [N][Ho][Wo] */
    float *tcoh;         /* [Ho][Wo] or NULL */
    uint8_t *status;     /* [Ho][Wo] */
} plk_stack_desc;

typedef struct plk_batch plk_batch;

/* A batch runs S1-S6 (Sec. III-A, II-A, III-B, III-C) for many independent
 * stacks of uneven length N with one window: for each stack, amplitude sums
 * over its N dates, GLRT SHP selection with n_eff = N, coherence, EMI with its
 * ref_idx, gamma_t -- the same results as plk_phase_link_stack_noalloc (and as
 * plk_ministack_step on a fresh state for ref_idx = 0).  The paper processes
 * bursts one after another; this serves many bursts, or many small
 * mini-stacks, in one call.  plk_batch_create checks the descriptors, copies
 * them and allocates every stack's scratch (sums, masks, counts, coherence, a
 * re-solve counter); the caller's arrays must stay valid until
 * plk_batch_destroy.  Errors: EINVAL (bad descriptor or window, with the
 * stack index), EUNSUPPORTED (bfloat16 coherence with N > 32), ENOMEM, ECUDA. */
plk_status plk_batch_create(plk_ctx *ctx, const plk_stack_desc *stacks, int n_stacks, plk_window win,
                            const plk_params *params, plk_batch **out);
/* Run every stack.  The first call tunes the launch schedule for each
 * distinct (N, window) not yet tuned in ctx (it times candidate coherence
 * tiles and EMI lanes per pixel on the batch's own data, so that call runs
 * the stages several times and waits for them), then records the whole batch
 * -- stacks spread over several streams, longest first -- as one CUDA graph;
 * every call (the first included) then launches that graph on ctx's stream.
 * Errors: ECUDA (with the failing stage), EINVAL. */
plk_status plk_batch_run(plk_ctx *ctx, plk_batch *b);
/* graph_built: 1 once recorded; streams: branches of the graph; nodes: graph
 * nodes (kernels and dependencies). */
plk_status plk_batch_info(const plk_batch *b, int *graph_built, int *streams, int *nodes);
plk_status plk_batch_destroy(plk_batch *b);
/* The schedule the autotuner chose for (N, window) in ctx: coherence tile
 * (output pixels) and the EMI row length (8, 16, 20, 24, 28 or 32 entries:
 * the smallest that holds N or the next; 8 and 16 are lanes per pixel, the
 * others run one pixel a warp); EINVAL if not tuned. */
plk_status plk_tuned_schedule(const plk_ctx *ctx, int N, plk_window win, int *cov_tile_y, int *cov_tile_x,
                              int *emi_lanes);

/* ------------------------------------------------------ spatial tiles */

/* One spatial tile of a burst, for independent processes (one per GPU or per
 * job; the path needs no exchange between them).  Output pixels depend only on
 * the samples of their SHP window (Sec. III-A) and, along the sequential chain,
 * on the compressed SLCs of earlier mini-stacks in that window (Sec. II-B), so
 * a tile is processed from an input crop that holds its cells' windows: a
 * read-only halo, one window wider for every further mini-stack step.
 *   y0, x0, h, w      the input crop: burst rows y0 .. y0+h-1, columns
 *                     x0 .. x0+w-1 (y0, x0 multiples of the strides, so the
 *                     crop's output cells are the burst's);
 *   oy0, ox0, oh, ow  the owned output cells of the burst's grid;
 *   cy0, cx0          where the owned cells sit in the crop's output grid
 *                     (burst cell oy0 + i is crop cell cy0 + i);
 *   py0, px0, ph, pw  the owned full-resolution pixels: the owned cells'
 *                     decimation blocks (the last cell row/column's running
 *                     to the image end), where the crop's compressed SLC
 *                     equals the burst's. */
typedef struct plk_tile {
    int32_t y0, x0, h, w;
    int32_t oy0, ox0, oh, ow;
    int32_t cy0, cx0;
    int32_t py0, px0, ph, pw;
} plk_tile;
/* Split the Ho x Wo output grid of an H x W burst into tiles_y x tiles_x tiles
 * of near-equal cell counts (tiles[ty * tiles_x + tx], host memory) and give
 * each the smallest crop, grown a stride at a time, on which a state that
 * runs `steps` mini-stack steps (plk_ministack_step on the crops of the same
 * SLCs, same window and parameters) produces, on the owned cells, the burst's
 * phases, gamma_t, statuses and SHP counts at every step, and on the owned
 * pixels its compressed SLCs (a cell is exact when its window, clipped to the
 * burst, lies in the crop, its decimation block is the same in both, and its
 * window's compressed SLCs were exact at every earlier step).  Host only.
 * Errors: EINVAL (no tiles, more tiles than output cells along an axis,
 * steps outside 1..256, bad window). */
plk_status plk_tile_plan(int H, int W, plk_window win, int tiles_y, int tiles_x, int steps, plk_tile *tiles);

/* ------------------------------------------- allocation-free variant */

/* Scratch capacity of plk_phase_link_stack_noalloc, in bytes: one array of
 * this size is held on every device that loads the library, until exit. */
#define PLK_NOALLOC_SCRATCH_BYTES (32u << 20)

/* One mini-stack of N real SLCs slc [N][H][W] through S1-S6 (amplitude sums,
 * GLRT SHP with n_eff = N, coherence, EMI with reference ref_idx, gamma_t)
 * without allocating any device memory.  No counterpart in the paper: this is
 * for callers that cannot call cudaMalloc, for example a plug-in running
 * inside a host application that owns every device allocation, or a service
 * that must not allocate after start-up.  Outputs as plk_phase_link:
 * phase [N][Ho][Wo], tcoh and status [Ho][Wo]; shp_count [Ho][Wo] may be NULL.
 * Results equal those of plk_ministack_step on a fresh state (ref_idx = 0)
 * with the same params; coherence in FP32, BF16 or FP16 (params->cov_precision,
 * N <= 32 for the last two).  Persistent-scatterer regridding
 * (params->ps_da_max > 0) is not run here: EUNSUPPORTED.  params are checked
 * as by the other entry points (EINVAL).
 * Work is issued on cuda_stream on the CURRENT device.
 * Scratch: sums, masks, counts and coherence live in a file-scope device array
 * of PLK_NOALLOC_SCRATCH_BYTES shared by every call; inputs and outputs stay
 * the caller's.  A request needing more (about 1 KB per output pixel at N=15
 * plus 4 bytes per input pixel) returns PLK_EINVAL with the sizes in
 * plk_last_error(NULL).  Every scratch region is written in full before it is
 * read within a call, so nothing needs clearing; calls that overlap on the
 * GPU (other streams, other threads) race on the shared array and must be
 * serialized by the caller.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, so the address is right even
 * after that device's context was reset and made again; the first call on a
 * device also loads the library's device code there, so make that first call
 * before any stream capture.  Errors: EINVAL (bad argument, too large),
 * EUNSUPPORTED, ECUDA; text in plk_last_error(NULL). */
plk_status plk_phase_link_stack_noalloc(const plk_c64 *slc, int N, int H, int W, plk_window win,
                                        int ref_idx, const plk_params *params, float *phase,
                                        float *tcoh, uint8_t *status, uint16_t *shp_count,
                                        void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PLK_H_ */
