"""Pins for the oracle's exponentially weighted merged amplitude statistics
(Sec. III-A, eqs. (merged-mean), (merged-variance), the exponential-decay
weighting option).

* lam = 1 is the equal-weight option: the sums equal the C oracle's
  accumulated single-precision sums, W1 = W2 = n and nu = n.
* Merging group by group equals the weighted sum over all images at once
  (the recursion is the definition unrolled), for uneven groups.
* A pixel of constant amplitude has that mean and zero variance, whatever
  the weights; the variance is never negative.
* The newest image weighs 1, each older one lam times the next; lam -> 0
  leaves one effective look.
* The real-valued F threshold equals the C oracle's bisection at integer
  looks, and decreases as the number of looks grows.
"""
import numpy as np
import pytest

import oracle


def stack(n, H=6, W=7, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, H, W)) + 1j * rng.standard_normal((n, H, W))).astype(np.complex64)


def test_equal_weights_reproduce_the_plain_sums():
    groups = [stack(5, seed=1), stack(3, seed=2), stack(7, seed=3)]
    st = None
    for g in groups:
        st = oracle.merge_group(st, g, 1.0)
    sp, sa = None, None
    for i, g in enumerate(groups):
        sp, sa = oracle.amp_stats(g, sp, sa, accumulate=i > 0)
    np.testing.assert_allclose(st["P"], sp, rtol=1e-5)
    np.testing.assert_allclose(st["A"], sa, rtol=1e-5)
    assert st["W1"] == 15 and st["W2"] == 15 and oracle.effective_looks(st) == 15


@pytest.mark.parametrize("lam", [0.5, 0.9, 0.99])
def test_group_merges_equal_the_direct_weighted_sum(lam):
    groups = [stack(4, seed=4), stack(1, seed=5), stack(6, seed=6)]
    st = None
    for g in groups:
        st = oracle.merge_group(st, g, lam)
    z = np.concatenate(groups).astype(np.complex128)
    w = oracle.decay_weights(z.shape[0], lam)
    np.testing.assert_allclose(st["P"], np.tensordot(w, np.abs(z) ** 2, axes=1), rtol=1e-12)
    np.testing.assert_allclose(st["A"], np.tensordot(w, np.abs(z), axes=1), rtol=1e-12)
    assert st["W1"] == pytest.approx(w.sum(), rel=1e-12)
    assert st["W2"] == pytest.approx((w * w).sum(), rel=1e-12)
    assert 1.0 <= oracle.effective_looks(st) <= z.shape[0]


def test_constant_amplitude_and_nonnegative_variance():
    rng = np.random.default_rng(7)
    a = rng.uniform(0.5, 2.0, (5, 6))
    z = a[None] * np.exp(1j * rng.uniform(-np.pi, np.pi, (9, 5, 6)))
    st = oracle.merge_group(oracle.merge_group(None, z[:4], 0.8), z[4:], 0.8)
    mu, var = oracle.merged_mean_variance(st)
    np.testing.assert_allclose(mu, a, rtol=1e-12)
    np.testing.assert_allclose(var, 0.0, atol=1e-12)
    st2 = oracle.merge_group(None, stack(12, seed=8), 0.7)
    assert np.all(oracle.merged_mean_variance(st2)[1] >= -1e-12)


def test_weights_and_effective_looks_limits():
    w = oracle.decay_weights(5, 0.5)
    np.testing.assert_array_equal(w, [0.0625, 0.125, 0.25, 0.5, 1.0])
    st = oracle.merge_group(None, stack(20, seed=9), 1e-6)
    assert oracle.effective_looks(st) == pytest.approx(1.0, abs=1e-5)


@pytest.mark.parametrize("n", [2, 10, 15, 30])
def test_real_threshold_matches_the_integer_bisection(n):
    assert oracle.glrt_threshold_real(1e-3, n) == pytest.approx(oracle.glrt_threshold(1e-3, n), rel=1e-8)
    assert oracle.glrt_threshold_real(1e-3, n + 0.5) < oracle.glrt_threshold_real(1e-3, n)


# ------------------------------------------------ single-precision decision sums

def test_f32_sums_at_equal_weights_are_the_plain_sums_bit_for_bit():
    """lam = 1: every weight is exactly 1, so the decision-precision merge is
    the C oracle's equal-weight accumulation, bit for bit."""
    groups = [stack(5, seed=11), stack(2, seed=12), stack(9, seed=13)]
    P = A = None
    sp = sa = None
    for i, g in enumerate(groups):
        P, A = oracle.merge_group_f32(P, A, g, 1.0)
        sp, sa = oracle.amp_stats(g, sp, sa, accumulate=i > 0)
    assert P.dtype == np.float32 and np.array_equal(P, sp) and np.array_equal(A, sa)


@pytest.mark.parametrize("lam", [0.5, 0.9, 0.97])
def test_f32_sums_follow_the_double_sums(lam):
    groups = [stack(6, seed=14), stack(3, seed=15), stack(4, seed=16)]
    st = None
    P = A = None
    for g in groups:
        st = oracle.merge_group(st, g, lam)
        P, A = oracle.merge_group_f32(P, A, g, lam)
    np.testing.assert_allclose(P, st["P"], rtol=2e-6)
    np.testing.assert_allclose(A, st["A"], rtol=2e-6)


@pytest.mark.parametrize("lam", [0.6, 0.95, 1.0])
def test_weight_sums_and_step_weights(lam):
    w, s = oracle.step_weights(5, lam)
    assert w[-1] == 1.0 and w.dtype == np.float32
    np.testing.assert_allclose(w[:-1] / w[1:], lam, rtol=1e-6)
    assert s == pytest.approx(lam ** 5, rel=1e-6)
    st, ws = None, None
    for M in (4, 7, 2):
        st = oracle.merge_group(st, stack(M, seed=M), lam)
        ws = oracle.weight_sums(ws, M, lam)
    assert ws[0] == pytest.approx(st["W1"], rel=1e-6) and ws[1] == pytest.approx(st["W2"], rel=1e-6)
    if lam == 1.0:
        assert ws == (13.0, 13.0)
