"""Sample coherence with real per-sample window weights, oracle side (Sec. II-A,
eq. (sample-coherence), the SHP mask of Sec. III-A read as weights).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For output pixel p with window samples z(q_b), b = 0 .. wy*wx - 1 in row-major
window order, and real weights w_b:

    S = sum_b w_b z(q_b) z(q_b)^H,      C_ik = S_ik / sqrt(S_ii S_kk).

With w the 0/1 SHP mask this is the estimator of Sec. II-A over the SHP set;
scaling every w_b by one factor leaves C unchanged.  Samples outside the image
are left out.  Plain double precision, one pixel at a time.
"""
from __future__ import annotations

import numpy as np


def window_samples(z: np.ndarray, window, oy: int, ox: int) -> tuple[np.ndarray, np.ndarray]:
    """Samples [wy*wx, N] of output pixel (oy, ox) (0 outside the image) and
    whether each lies inside the image."""
    wy, wx, sy, sx = window
    N, H, W = z.shape
    cy, cx = oy * sy + sy // 2, ox * sx + sx // 2
    out = np.zeros((wy * wx, N), np.complex128)
    inside = np.zeros(wy * wx, bool)
    b = 0
    for dy in range(-(wy // 2), wy // 2 + 1):
        for dx in range(-(wx // 2), wx // 2 + 1):
            y, x = cy + dy, cx + dx
            if 0 <= y < H and 0 <= x < W:
                out[b] = z[:, y, x]
                inside[b] = True
            b += 1
    return out, inside


def weighted_coherence(samples: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """Packed upper triangle (row-major, i <= k) of C from samples [nb, N] and weights [nb]."""
    zs = np.asarray(samples, dtype=np.complex128)
    w = np.asarray(weights, dtype=np.float64)
    S = (zs.T * w) @ zs.conj()                 # S_ik = sum_b w_b z_i(b) conj(z_k(b))
    d = np.sqrt(np.real(np.diag(S)))
    C = S / np.outer(d, d)
    N = S.shape[0]
    return np.concatenate([C[i, i:] for i in range(N)])


def mask_weights(mask_words: np.ndarray, nb: int) -> np.ndarray:
    """The 0/1 weights [nb] of one pixel's mask words (bit b of word b // 64)."""
    words = np.asarray(mask_words, dtype=np.uint64)
    return np.array([float((int(words[b // 64]) >> (b % 64)) & 1) for b in range(nb)])
