"""Phase cosine similarity gamma_s of the oracle (Sec. III-C, eq. (phase-cosine-sim)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a pixel p with linked phases phi_hat (its M real dates) and a neighbour x
in the search window W, the similarity is the mean, over the N_ifg
interferograms of the re-formed network, of cos(phi_hat_ifg - x_ifg), the
interferogram phases being phase(b) - phase(a) for each pair (a, b) of the
network.  gamma_s(p) is the median of these similarities over x in W.

Readings (the paper leaves them open):
* network: the nearest-3 network of Sec. III-D, every pair (a, b) of real dates
  with 1 <= b - a <= 3 (3M - 6 interferograms for M >= 3; M - 1 + ... for less);
* W: the disk of radius r output pixels, dy^2 + dx^2 <= r^2, without p itself;
  neighbours outside the image or with a non-finite phase are left out;
* median of an even count: the mean of the two middle values;
* p with a non-finite phase, or without any neighbour left: NaN.
Plain double precision, vectorised over pixels one window offset at a time.
"""
from __future__ import annotations

import numpy as np


def nearest3_pairs(M: int) -> list[tuple[int, int]]:
    """Interferogram pairs (a, b), a < b, of the nearest-3 network over M dates."""
    return [(a, a + d) for d in (1, 2, 3) for a in range(M - d)]


def disk_offsets(r: int) -> list[tuple[int, int]]:
    """Window offsets (dy, dx) with 0 < dy^2 + dx^2 <= r^2."""
    return [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if 0 < dy * dy + dx * dx <= r * r]


def phase_similarity(phase: np.ndarray, radius: int) -> np.ndarray:
    """gamma_s [Ho, Wo] (float64) of linked phases phase [M, Ho, Wo]."""
    ph = np.asarray(phase, dtype=np.float64)
    M, Ho, Wo = ph.shape
    assert M >= 2 and radius >= 1
    pairs = nearest3_pairs(M)
    a = np.array([p[0] for p in pairs])
    b = np.array([p[1] for p in pairs])
    ifg = ph[b] - ph[a]                                     # [N_ifg, Ho, Wo]
    valid = np.all(np.isfinite(ph), axis=0)
    offs = disk_offsets(radius)
    sims = np.full((len(offs), Ho, Wo), np.nan)
    for j, (dy, dx) in enumerate(offs):
        # centre rows/cols whose neighbour (y + dy, x + dx) is inside the image
        y0, y1 = max(0, -dy), min(Ho, Ho - dy)
        x0, x1 = max(0, -dx), min(Wo, Wo - dx)
        if y0 >= y1 or x0 >= x1:
            continue
        cen = ifg[:, y0:y1, x0:x1]
        nb = ifg[:, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        s = np.mean(np.cos(cen - nb), axis=0)               # the similarity of eq. (phase-cosine-sim)
        s[~valid[y0 + dy:y1 + dy, x0 + dx:x1 + dx]] = np.nan
        sims[j, y0:y1, x0:x1] = s
    out = np.full((Ho, Wo), np.nan)
    have = np.any(np.isfinite(sims), axis=0) & valid
    if np.any(have):
        out[have] = np.nanmedian(sims[:, have], axis=0)
    return out
