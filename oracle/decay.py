"""Merged amplitude statistics with exponentially decaying image weights,
oracle side (Sec. III-A, eqs. (merged-mean) and (merged-variance), the second
weighting option the paper names beside equal weights per image).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the paper names the option without a formula):
* image t of T seen so far (t = 0 oldest) has weight w_t = lam^(T - 1 - t),
  0 < lam <= 1, so the newest image weighs 1 and lam = 1 is the equal-weight
  option;
* a new group of M images merges into the running sums as
  S <- lam^M S + sum_j lam^(M - 1 - j) s_j  for S in (sum |z|^2, sum |z|, W1),
  and W2 (the sum of squared weights) with lam^(2M) and lam^(2(M - 1 - j));
* merged mean amplitude mu = sum_t w_t |z_t| / W1 and merged second moment
  sum_t w_t |z_t|^2 / W1, so eq. (merged-variance) reads
  sigma^2 = sum_t w_t |z_t|^2 / W1 - mu^2;
* the GLRT of Sec. III-A compares two pixels' weighted power sums; with
  unequal weights a weighted sum of exponential variables is no longer a
  scaled chi-square, and the test uses the effective number of looks
  nu = W1^2 / W2 in place of n (nu = n for equal weights): accept q iff
  max(P_p, P_q) <= c min(P_p, P_q), c = F^{-1}_{2 nu, 2 nu}(1 - alpha / 2).
Plain double precision; scipy's F quantile as a step.
"""
from __future__ import annotations

import numpy as np
import scipy.stats


def decay_weights(n_images: int, lam: float) -> np.ndarray:
    """w_t = lam^(n - 1 - t), t = 0 (oldest) .. n - 1 (newest)."""
    return lam ** (n_images - 1 - np.arange(n_images, dtype=np.float64))


def merge_group(state: dict | None, group: np.ndarray, lam: float) -> dict:
    """Merge a group of images [M, H, W] (oldest first) into the running sums."""
    z = np.asarray(group, dtype=np.complex128)
    M = z.shape[0]
    w = decay_weights(M, lam)
    amp = np.abs(z)
    new = {"P": np.tensordot(w, amp ** 2, axes=1), "A": np.tensordot(w, amp, axes=1),
           "W1": float(w.sum()), "W2": float((w * w).sum()), "n": M}
    if state is None:
        return new
    s = lam ** M
    return {"P": s * state["P"] + new["P"], "A": s * state["A"] + new["A"], "W1": s * state["W1"] + new["W1"],
            "W2": s * s * state["W2"] + new["W2"], "n": state["n"] + M}


def merged_mean_variance(state: dict) -> tuple[np.ndarray, np.ndarray]:
    """Weighted mean amplitude and variance, eqs. (merged-mean), (merged-variance)."""
    mu = state["A"] / state["W1"]
    return mu, state["P"] / state["W1"] - mu * mu


def effective_looks(state: dict) -> float:
    """nu = W1^2 / W2."""
    return state["W1"] ** 2 / state["W2"]


def glrt_threshold_real(alpha: float, nu: float) -> float:
    """c = F^{-1}_{2 nu, 2 nu}(1 - alpha / 2) for a real number of looks."""
    return float(scipy.stats.f.ppf(1.0 - alpha / 2.0, 2.0 * nu, 2.0 * nu))
