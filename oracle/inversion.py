"""L1 time-series network inversion by ADMM, oracle side (Sec. III-E,
eq. (l1-min); Appendix, "Details on ADMM Algorithm for L1 Minimization").

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per pixel, with b the unwrapped interferogram phases of the network and A the
incidence matrix (row (a, b): -1 at date a, +1 at date b, date 0 dropped, so
x is the phase relative to the first date), minimise ||A x - b||_1 by

    x^{k+1} = (A^T A)^{-1} A^T (b + z^k - u^k)
    z^{k+1} = S_{1/rho}(A x^{k+1} - b + u^k)
    u^{k+1} = u^k + A x^{k+1} - b - z^{k+1}

with S the soft-thresholding operator, the Cholesky factor of A^T A shared by
all pixels.  Readings: z^0 = u^0 = 0; a fixed number of iterations (the paper
states no stopping rule); rho a parameter.  Plain double precision, numpy and
scipy's Cholesky routines as steps.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def incidence(pairs, n_dates: int) -> np.ndarray:
    """A [N_ifg, n_dates - 1] of the network `pairs` ((a, b), a < b)."""
    A = np.zeros((len(pairs), n_dates - 1))
    for k, (a, b) in enumerate(pairs):
        if a > 0:
            A[k, a - 1] = -1.0
        if b > 0:
            A[k, b - 1] = 1.0
    return A


def soft_threshold(a: np.ndarray, kappa: float) -> np.ndarray:
    """S_kappa(a): a - kappa above kappa, a + kappa below -kappa, 0 between."""
    return np.where(a > kappa, a - kappa, np.where(a < -kappa, a + kappa, 0.0))


def l1_invert(b: np.ndarray, pairs, n_dates: int, rho: float, iters: int) -> dict:
    """ADMM on every pixel of b [N_ifg, npx]: x [n_dates-1, npx], residual b - A x."""
    b = np.asarray(b, dtype=np.float64)
    A = incidence(pairs, n_dates)
    cho = scipy.linalg.cho_factor(A.T @ A, lower=True)      # once for all pixels
    z = np.zeros_like(b)
    u = np.zeros_like(b)
    x = np.zeros((A.shape[1], b.shape[1]))
    for _ in range(iters):
        x = scipy.linalg.cho_solve(cho, A.T @ (b + z - u))
        Ax = A @ x
        z = soft_threshold(Ax - b + u, 1.0 / rho)
        u = u + Ax - b - z
    return {"x": x, "residual": b - A @ x}
