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


def step_weights(M: int, lam: float) -> tuple[np.ndarray, np.float32]:
    """The weights of one merge in single precision: w_j = lam^(M - 1 - j)
    for the group's images j = 0..M-1 and s = lam^M for the running sums,
    each a product of lam's formed in double precision (w_{M-1} = 1, w_{j-1} =
    w_j lam, s = w_0 lam) and rounded once to single precision."""
    w = np.empty(M, np.float64)
    acc = 1.0
    for j in range(M - 1, -1, -1):
        w[j] = acc
        acc *= lam
    return w.astype(np.float32), np.float32(acc)


def merge_group_f32(sum_pow: np.ndarray | None, sum_amp: np.ndarray | None, group: np.ndarray, lam: float):
    """merge_group's sums P and A in single precision, in the fixed order the
    GLRT decision is taken in on both sides of the parity test (the paper
    fixes no precision for it): per pixel, q_j = fl(fl(x^2) + fl(y^2)) and
    P_g = sum_j fl(w_j q_j), A_g = sum_j fl(w_j sqrt(q_j)), j ascending from 0;
    then P = fl(fl(s P_old) + P_g), A likewise (P = P_g on a first group).  With
    lam = 1 every weight is 1 and this is the equal-weight sum of amp_stats.
    Returns new float32 arrays."""
    z = np.asarray(group, dtype=np.complex64)
    M = z.shape[0]
    w, s = step_weights(M, lam)
    Pg = np.zeros(z.shape[1:], np.float32)
    Ag = np.zeros(z.shape[1:], np.float32)
    for j in range(M):
        x, y = z[j].real.astype(np.float32), z[j].imag.astype(np.float32)
        q = (x * x) + (y * y)
        Pg = Pg + w[j] * q
        Ag = Ag + w[j] * np.sqrt(q)
    if sum_pow is None:
        return Pg, Ag
    return (s * np.asarray(sum_pow, np.float32)) + Pg, (s * np.asarray(sum_amp, np.float32)) + Ag


def weight_sums(prev: tuple[float, float] | None, M: int, lam: float) -> tuple[float, float]:
    """W1 = sum of weights and W2 = sum of squared weights after merging a
    group of M images into running sums (W1, W2) (None: the first group), in
    double precision with the same single-precision weights as the sums."""
    w, s = step_weights(M, lam)
    w1 = float(np.sum(w.astype(np.float64)))
    w2 = float(np.sum(w.astype(np.float64) ** 2))
    if prev is None:
        return w1, w2
    W1, W2 = prev
    sd = float(s)
    return sd * W1 + w1, sd * sd * W2 + w2


def glrt_threshold_real(alpha: float, nu: float) -> float:
    """c = F^{-1}_{2 nu, 2 nu}(1 - alpha / 2) for a real number of looks."""
    return float(scipy.stats.f.ppf(1.0 - alpha / 2.0, 2.0 * nu, 2.0 * nu))
