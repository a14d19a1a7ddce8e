"""Pins for the oracle's L1 network inversion by ADMM (Sec. III-E,
eq. (l1-min); Appendix).

* The incidence matrix of a small network written out; the soft-thresholding
  operator's three branches.
* Without unwrapping errors (b = A x) the true x is a fixed point reached in
  one iteration from z = u = 0.
* With sparse 2 pi unwrapping errors, the iterates recover the true x and the
  residual is exactly the injected 2 pi k (the L1 minimiser, Sec. III-E).
* On noisy b, the objective ||A x - b||_1 after many iterations matches the
  optimum of the same problem solved as a linear programme by scipy's HiGHS
  (an independent solver).
* Equivariance: b + A c gives x + c at every iteration.
"""
import numpy as np
import pytest
import scipy.optimize

import oracle


def test_incidence_matrix_written_out():
    A = oracle.incidence([(0, 1), (1, 2), (0, 2), (1, 3)], 4)
    want = np.array([[1, 0, 0], [-1, 1, 0], [0, 1, 0], [-1, 0, 1]], float)
    assert np.array_equal(A, want)
    x = np.array([0.5, -1.0, 2.0])                          # dates 1..3 relative to date 0
    assert np.allclose(A @ x, [0.5, -1.5, -1.0, 1.5])


def test_soft_threshold_branches():
    a = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    assert np.array_equal(oracle.soft_threshold(a, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0])


def true_series(n_dates, npx, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0, 2.0, (n_dates - 1, npx)), axis=0)


def test_consistent_phases_are_a_fixed_point():
    pairs = oracle.nearest3_pairs(15)
    A = oracle.incidence(pairs, 15)
    xt = true_series(15, 20, 0)
    o = oracle.l1_invert(A @ xt, pairs, 15, rho=1.0, iters=1)
    np.testing.assert_allclose(o["x"], xt, atol=1e-12)
    np.testing.assert_allclose(oracle.l1_invert(A @ xt, pairs, 15, 1.0, 30)["x"], xt, atol=1e-12)


@pytest.mark.parametrize("rho", [0.5, 1.0, 2.0])
def test_sparse_unwrapping_errors_are_rejected(rho):
    n, npx = 15, 40
    pairs = oracle.nearest3_pairs(n)
    A = oracle.incidence(pairs, n)
    xt = true_series(n, npx, 1)
    rng = np.random.default_rng(2)
    k = np.zeros((len(pairs), npx))
    for p in range(npx):                                   # one or two wrong interferograms per pixel
        idx = rng.choice(len(pairs), size=1 + p % 2, replace=False)
        k[idx, p] = rng.choice([-2, -1, 1, 2], size=idx.size)
    o = oracle.l1_invert(A @ xt + 2 * np.pi * k, pairs, n, rho, 300)
    np.testing.assert_allclose(o["x"], xt, atol=1e-6)
    np.testing.assert_allclose(o["residual"], 2 * np.pi * k, atol=1e-5)


def lp_optimum(A, b):
    """min sum(t) s.t. -t <= A x - b <= t, as a linear programme (HiGHS)."""
    m, n = A.shape
    c = np.concatenate([np.zeros(n), np.ones(m)])
    A_ub = np.block([[A, -np.eye(m)], [-A, -np.eye(m)]])
    b_ub = np.concatenate([b, -b])
    res = scipy.optimize.linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * n + [(0, None)] * m,
                                 method="highs")
    assert res.status == 0
    return res.fun


def test_objective_matches_the_linear_programme():
    n, npx = 10, 6
    pairs = oracle.nearest3_pairs(n)
    A = oracle.incidence(pairs, n)
    rng = np.random.default_rng(3)
    b = A @ true_series(n, npx, 4) + rng.normal(0, 0.8, (len(pairs), npx))
    o = oracle.l1_invert(b, pairs, n, rho=1.0, iters=3000)
    for p in range(npx):
        got = np.abs(A @ o["x"][:, p] - b[:, p]).sum()
        best = lp_optimum(A, b[:, p])
        assert got <= best * (1 + 1e-4) + 1e-9, (p, got, best)


def test_equivariance_to_consistent_shifts():
    n = 12
    pairs = [(a, b) for (a, b) in oracle.nearest3_pairs(n) if b - a <= 2]   # a nearest-2 sub-network
    A = oracle.incidence(pairs, n)
    rng = np.random.default_rng(5)
    b = A @ true_series(n, 8, 6) + rng.normal(0, 1.0, (len(pairs), 8))
    c = rng.normal(0, 3.0, (n - 1, 1))
    for iters in (1, 7, 40):
        o1 = oracle.l1_invert(b, pairs, n, 1.0, iters)
        o2 = oracle.l1_invert(b + A @ c, pairs, n, 1.0, iters)
        np.testing.assert_allclose(o2["x"], o1["x"] + c, atol=1e-9)


@pytest.mark.parametrize("rho,want", [(2.0, 2.0 / 3.0), (0.5, 1.0)])
def test_two_iterations_by_hand(rho, want):
    # Three copies of one interferogram with b = (0, 0, 3): the L1 answer is the
    # median 0, least squares the mean 1.  From z = u = 0: x1 = 1; r = A x1 - b =
    # (1, 1, -2); z1 = S_{1/rho}(r); u1 = r - z1; x2 = mean(b + z1 - u1) =
    # 1 + (2/3) sum(z1).  rho = 2: z1 = (0.5, 0.5, -1.5), x2 = 2/3;  rho = 0.5:
    # z1 = 0, x2 = 1 (a threshold of rho instead of 1/rho would swap them).
    b = np.array([[0.0], [0.0], [3.0]])
    o1 = oracle.l1_invert(b, [(0, 1)] * 3, 2, rho, 1)
    o2 = oracle.l1_invert(b, [(0, 1)] * 3, 2, rho, 2)
    assert abs(o1["x"][0, 0] - 1.0) < 1e-12
    assert abs(o2["x"][0, 0] - want) < 1e-12
