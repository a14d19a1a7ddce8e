// Internal declarations shared by the CUDA translation units of libplk.
// Kernels are written for sm_103a (GB300).  Nothing here is part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "plk.h"

namespace plk {

// Date planes of one mini-stack.  The planes of compressed SLCs (ring order)
// and of the new real SLCs live in different buffers, so kernels receive one
// base pointer per mini-stack entry, read from the parameter space.
struct Planes {
    const float2 *p[PLK_MAX_N];
};

struct Geom {
    int H, W;        // input image
    int wy, wx;      // window (odd)
    int hy, hx;      // half window
    int sy, sx;      // output strides
    int Ho, Wo;      // output grid
    int nwords;      // uint64 mask words per output pixel
};

inline Geom make_geom(int H, int W, plk_window w) {
    Geom g;
    g.H = H; g.W = W; g.wy = w.wy; g.wx = w.wx; g.hy = w.wy / 2; g.hx = w.wx / 2;
    g.sy = w.sy; g.sx = w.sx; g.Ho = H / w.sy; g.Wo = W / w.sx;
    g.nwords = (w.wy * w.wx + 63) / 64;
    return g;
}

// Parameters of the phase-linking kernels, resolved on the host.
struct EmiParams {
    float beta, mu, tol, cond_max, err_max;
    int max_iter;
    int fp64_resolve;
    unsigned long long *work;  // device work area of the FP64 re-solve, kEmiWorkBytes (owned by the caller)
};

// Work area of one phase-link launch pair: counter 0 is the re-solve's chunk
// cursor over the status array, counter 1 the length of the pending list the
// single-precision pass appends to, counter 2 the re-solve's cursor in that
// list; the list (kPendCap pixel indices) starts at byte 256.  A longer
// pending set overflows the list and the re-solve scans the statuses instead.
constexpr int kPendCap = 65536;
constexpr size_t kEmiWorkBytes = 256 + (size_t)kPendCap * sizeof(unsigned);
__host__ __device__ inline unsigned *pending_list(unsigned long long *work) {
    return reinterpret_cast<unsigned *>(reinterpret_cast<char *>(work) + 256);
}

__host__ __device__ inline long long ntri(int n) { return (long long)n * (n + 1) / 2; }
__host__ __device__ inline int packed_index(int n, int i, int k) { return i * n - i * (i - 1) / 2 + (k - i); }

// ---------------------------------------------------------------- launches
// Each returns cudaGetLastError() after the launch.
// z: n contiguous planes of npix samples.
// PS outputs of S1: D_A of the merged sums over n_eff images per pixel where
// it is at most 1.001 da_max (+inf above that, where a new sample is zero or
// where the amplitude sum is 0), and where D_A <= da_max the sum of |z| over
// the new images (elsewhere amp_new is not written).
struct PsStats {
    float *da = nullptr, *amp_new = nullptr;
    float n_eff = 0.f, da_max = 0.f;
};
// Weights of a decaying merge: image j of the new group weighs w[j], the
// running sums are scaled by s before the group is added.
struct SumWeights {
    float w[PLK_MAX_N] = {};
    float s = 1.f;
};
cudaError_t launch_amp_stats(const float2 *z, int n, long long npix, float *sum_pow, float *sum_amp,
                             int accumulate, cudaStream_t s, const PsStats *ps = nullptr,
                             const SumWeights *wts = nullptr);
cudaError_t launch_shp(const float *sum_pow, const Geom &g, float c, uint64_t *mask, uint16_t *count,
                       cudaStream_t s);
// Returns cudaErrorInvalidConfiguration if the window/N combination exceeds
// shared memory even at a 1x1 output tile.
// Launch schedule chosen by the batch autotuner (0 = the built-in heuristic).
// Row length of the EMI kernels for n dates: the smallest of 8 and 16 (four
// and two pixels a warp, NP lanes each) and 20, 24, 28 and 32 (one pixel a
// warp) that holds n.  A solve costs about n times the row length, so the
// intermediate rows save padded work for 17 <= n <= 28.
__host__ __device__ inline int emi_row_length(int n) {
    return n <= 8 ? 8 : n <= 16 ? 16 : n <= 20 ? 20 : n <= 24 ? 24 : n <= 28 ? 28 : 32;
}

struct Schedule {
    int cov_TY = 0, cov_TX = 0;  // single-precision coherence tile (output pixels)
    int emi_np = 0;              // row length of the EMI kernels (emi_row_length values, >= n)
};

cudaError_t launch_covariance(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                              cudaStream_t s, int precision = 0, const Schedule *sch = nullptr);
// Up to max candidate single-precision coherence tiles {TY, TX} for (n, g),
// best heuristic score first; returns the count.
int covariance_tile_candidates(int n, const Geom &g, int (*tiles)[2], int max);
// precision 1: bfloat16 samples, tensor-core sums (n <= 32); precision 2:
// half-precision samples scaled by a power of two per tile, same sums.
cudaError_t launch_covariance_bf16(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                                   cudaStream_t s);
cudaError_t launch_covariance_fp16(const Planes &z, int n, const Geom &g, const uint64_t *mask, float2 *C,
                                   cudaStream_t s);
struct Prof;
// cudaMalloc that counts the library's device allocations (plk_device_allocations).
cudaError_t dev_malloc(void **p, size_t bytes);
extern std::atomic<long long> g_device_allocations;
// Where the double-precision re-solve recomputes a pixel's coherence from:
// the stack planes, geometry and SHP masks of the mini-stack.
struct StackSource {
    const Planes *z;
    const Geom *g;
    const uint64_t *mask;
};
cudaError_t launch_phase_link(const float2 *C, int n, long long npx, int ref, const EmiParams &prm,
                              float *phase, float *tcoh, float *lam, uint8_t *status, cudaStream_t s,
                              Prof *prof = nullptr, const StackSource *src = nullptr, const Schedule *sch = nullptr);
// Persistent-scatterer selection inputs: D_A per pixel as S1 writes it (+inf
// where a real sample is zero), the threshold and the mini-stack's reference
// entry (da == nullptr: off).
struct PsSelect {
    const float *da = nullptr, *amp_new = nullptr;  // as S1 writes them (PsStats)
    float da_max = 0.f;
    int ref = 0;
};
// shift_date >= 0: the phases are re-referenced to that date (its phase subtracted).
// ps on: each PS pixel is compressed on its own phases arg(z_i conj z_ref).
// Complex 16-bit samples (re, im interleaved) -> complex64, n samples; src
// and dst 16-byte aligned.
cudaError_t launch_ci16_to_c64(const int16_t *src, float2 *dst, long long n, cudaStream_t s);
cudaError_t launch_compress(const Planes &z, int n, int first_real, const Geom &g, const float *phase,
                            float2 *kappa, cudaStream_t s, int shift_date = -1, const PsSelect &ps = PsSelect());

// PS selection by amplitude dispersion and regridding onto the output grid:
// phase [n - first_real][Ho][Wo] and status [Ho][Wo] updated in place.  D_A
// from the merged sums (with the real samples checked), or, when da != nullptr,
// read from the plane S1 wrote (sum_pow, sum_amp unused).
cudaError_t launch_ps_regrid(const Planes &z, int n, int first_real, int ref, const Geom &g, const float *sum_pow,
                             const float *sum_amp, int n_eff, float da_max, float *phase, uint8_t *status,
                             cudaStream_t s, const float *da = nullptr);

// Phase cosine similarity gamma_s of linked phases [M][Ho][Wo] over a disk of
// radius r; cudaErrorInvalidConfiguration if no tile fits in shared memory.
cudaError_t launch_phase_similarity(const float *phase, int M, int Ho, int Wo, int r, float *gamma_s,
                                    cudaStream_t s);
int phase_sim_disk_count(int r);

// A network inside the nearest-3 network for the ADMM inversion over nxp
// unknown dates: slot admm_slot(nxp, d, a) holds pair (a, a + d), d <= 3,
// a + d <= nxp (3 nxp - 3 slots); plane[slot] is the caller's interferogram
// index (-1: not in the network).  L[i] =
// {1 / L_ii, L_i,i-1, L_i,i-2, L_i,i-3}: the banded Cholesky factor of A^T A
// (identity beyond nx).
struct AdmmNet {
    int plane[48];
    float L[16][4];
    float kappa;  // 1 / rho
    int iters, nx, nxp;
};
__host__ __device__ constexpr int admm_slot(int nxp, int d, int a) {
    return (d - 1) * nxp - (d - 1) * (d - 2) / 2 + a;
}
cudaError_t launch_admm_l1(const float *unw, long long npx, const AdmmNet &net, float *x, float *resid,
                           cudaStream_t s);

int device_sm_count();
// Nonzero if a bounded device-side wait gave up since the last call (then cleared).
// Adjoint of S3-S5 (masks frozen): scratch bytes and the launch sequence
// (coherence recomputed into the workspace).
size_t adjoint_workspace_bytes(int n, const Geom &g);
cudaError_t launch_adjoint(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                           const EmiParams &prm, const float *dphase, void *workspace, float2 *grad,
                           cudaStream_t s, Prof *prof = nullptr);
// Gradient of sum(dphase * phase) with respect to real window weights at the
// SHP mask, [Ho][Wo][wy*wx] (the adjoint's workspace).
cudaError_t launch_weight_gradient(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                                   const EmiParams &prm, const float *dphase, void *workspace, float *dw,
                                   cudaStream_t s);
// First-order standard deviation of the linked phases [n][Ho][Wo] under white
// circular noise of variance sigma2 on the samples (the adjoint's workspace).
cudaError_t launch_phase_uncertainty(const Planes &z, int n, const Geom &g, const uint64_t *mask, int ref,
                                     const EmiParams &prm, float sigma2, void *workspace, float *sd,
                                     cudaStream_t s);
int read_and_clear_wait_timeout();
cudaError_t launch_wait_selftest(cudaStream_t s);
// Text returned by plk_last_error(NULL) on this thread.
void set_noctx_error(const char *msg);

// Optional per-launch timing: events recorded on the launching stream around
// each kernel while enabled (see plk_profile_enable).
struct Prof {
    static constexpr int kMaxRecords = 4096;
    bool on = false;
    int n = 0;
    cudaEvent_t ev[2 * kMaxRecords] = {};
    const char *name[kMaxRecords] = {};
    bool overflow = false;
    void begin(const char *nm, cudaStream_t s) {
        if (!on) return;
        if (n >= kMaxRecords) { overflow = true; return; }
        name[n] = nm;
        cudaEventRecord(ev[2 * n], s);
    }
    void end(cudaStream_t s) {
        if (!on || n >= kMaxRecords) return;
        cudaEventRecord(ev[2 * n + 1], s);
        ++n;
    }
};

}  // namespace plk
