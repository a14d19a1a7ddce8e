"""Mini-stack chain of the oracle (Sec. II-B, "Proposed Approach"; Fig. 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each step, for new real SLCs z_1..z_M:
  1. merge amplitude statistics (Sec. III-A, eqs. (merged-mean), (merged-variance)
     with equal weight per image): P <- P + sum_t |z_t|^2, n <- n + M;
  2. GLRT SHP selection on P with n real samples per pixel (Sec. III-A);
  3. form the mini-stack [kappa ring oldest..newest, z_1..z_M] (Sec. II-B: the
     compressed SLCs are prepended; only the K most recent are kept);
  4. sample coherence over the SHP neighbourhood (eq. (sample-coherence));
  5. EMI phase linking with reference r = the newest compressed SLC, or the
     first real SLC when there is none (Sec. II-B items 1-3), and gamma_t;
  6. compress the real SLCs onto the linked phases (kappa = zeta^H z) and push
     kappa into the ring;
  7. with a PS threshold (Sec. IV; Supplement, "Regridding PS and DS"), output
     cells whose decimation block holds a PS take the phases of the one with
     the lowest amplitude dispersion, relative to the reference entry, and in
     step 6 each PS pixel is compressed on its own phases (PS are processed at
     full resolution), so kappa carries the PS's phase at the datum.
The phases returned for the real dates are relative to the first date of the
archive, because every kappa inherits the reference phase of the one before.

scheme="last" (the production variant of Sec. IV and the Supplement's
"Compressed SLC strategy for separate batched processing"): step 6 forms kappa
on the linked phases re-referenced to the mini-stack's last real SLC
(phase_i - phase_last), so kappa carries that date's phase and the next
mini-stack's phases are relative to it.
"""
from __future__ import annotations

import numpy as np

from . import amp_stats, compress, covariance, glrt_threshold, ntri, phase_link, ps_compress, ps_regrid, shp_select
from .decay import glrt_threshold_real, merge_group_f32, weight_sums


def ministack(z: np.ndarray, first_real: int, window, sum_pow: np.ndarray, n_eff: int,
              alpha: float, ref: int, beta: float = 0.0, cond: bool = False, scheme: str = "first",
              sum_amp: np.ndarray | None = None, ps_da_max: float = 0.0, c: float | None = None) -> dict:
    """One mini-stack through S2-S7 with statistics already merged (PS
    regridding of the returned phases when ps_da_max > 0).  c: the GLRT
    threshold, when it is not the one for n_eff looks (decaying weights)."""
    N = z.shape[0]
    if c is None:
        c = glrt_threshold(alpha, n_eff)
    mask, count = shp_select(sum_pow, window, np.float32(c))
    C = covariance(z, window, mask)
    out = phase_link(C, N, ref, beta, cond=cond)
    ph = out["phase"]
    if scheme == "last":
        ph = ph - ph[N - 1][None]  # re-referenced to the last real SLC
    kappa = compress(z, first_real, window, ph)
    has_cells = C.shape[0] * C.shape[1] > 0  # no output grid: nothing is linked, kappa stays 0
    if ps_da_max > 0 and has_cells:
        assert sum_amp is not None
        kappa = ps_compress(z, first_real, sum_pow, sum_amp, n_eff, ref, ps_da_max, kappa,
                            shift=N - 1 if scheme == "last" else -1)
    out.update(mask=mask, count=count, C=C, kappa=kappa, c=c)
    if ps_da_max > 0:
        real, st = ps_regrid(z, first_real, window, sum_pow, sum_amp, n_eff, ref, ps_da_max,
                             out["phase"][first_real:], out["status"])
        out["phase"] = np.concatenate([out["phase"][:first_real], real], axis=0)
        out["status"] = st
    return out


class OracleChain:
    """Sequential processing state: kappa ring, merged power sums, image count."""

    def __init__(self, H: int, W: int, window, K_max: int, alpha: float = 1e-3, beta: float = 0.0,
                 kappa_dtype=np.complex128, scheme: str = "first", ps_da_max: float = 0.0, decay: float = 1.0):
        assert scheme in ("first", "last")
        # decay < 1: step 1 merges with exponentially decaying image weights
        # (oracle/decay.py, single-precision sums in the decision order) and
        # step 2 takes nu = W1^2 / W2 effective looks.
        assert 0.0 < decay <= 1.0 and (decay == 1.0 or ps_da_max == 0.0)
        self.decay = decay
        self.wsum = None  # (W1, W2): sums of the image weights and of their squares
        self.scheme = scheme
        self.ps_da_max = ps_da_max
        # kappa_dtype=np.complex64 stores each compressed SLC rounded to the
        # single-precision complex samples a stored SLC has (the form the GPU
        # state keeps), so both sides can start a step from identical inputs.
        self.kappa_dtype = kappa_dtype
        self.H, self.W = H, W
        self.window = tuple(window)
        self.K_max = K_max
        self.alpha, self.beta = alpha, beta
        self.ring: list[np.ndarray] = []
        self.sum_pow = np.zeros((H, W), np.float32)
        self.sum_amp = np.zeros((H, W), np.float32)
        self.n = 0

    def step(self, new_slc: np.ndarray, cond: bool = False) -> dict:
        new_slc = np.ascontiguousarray(new_slc, dtype=np.complex64)
        M = new_slc.shape[0]
        c = None
        if self.decay == 1.0:
            amp_stats(new_slc, self.sum_pow, self.sum_amp, accumulate=True)
        else:
            first = self.n == 0
            self.sum_pow, self.sum_amp = merge_group_f32(None if first else self.sum_pow,
                                                         None if first else self.sum_amp, new_slc, self.decay)
            self.wsum = weight_sums(None if first else self.wsum, M, self.decay)
            c = glrt_threshold_real(self.alpha, max(1.0, self.wsum[0] ** 2 / self.wsum[1]))
        self.n += M
        K = len(self.ring)
        parts = [np.stack(self.ring).astype(np.complex128)] if K else []
        parts.append(new_slc.astype(np.complex128))
        z = np.concatenate(parts, axis=0)
        ref = K - 1 if K > 0 else 0
        out = ministack(z, K, self.window, self.sum_pow, self.n, self.alpha, ref, self.beta, cond, self.scheme,
                        self.sum_amp, self.ps_da_max, c)
        self.ring.append(out["kappa"].astype(self.kappa_dtype).astype(np.complex128))
        if len(self.ring) > self.K_max:
            self.ring.pop(0)
        out["phase_real"] = out["phase"][K:]
        out["K_used"] = K
        out["N"] = z.shape[0]
        return out


__all__ = ["OracleChain", "ministack", "ntri"]
