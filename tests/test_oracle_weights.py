"""Pins for the oracle's weighted sample coherence (Sec. II-A, eq.
(sample-coherence), the SHP mask of Sec. III-A read as real weights).

* At the 0/1 weights of an SHP mask it equals the C oracle's masked
  coherence (an independent implementation) at every output pixel, border
  pixels with samples outside the image included, for two window geometries.
* Scaling every weight by one factor leaves it unchanged; a zero weight is
  the same as leaving the sample out.
* A two-sample, two-date case written out by hand.
"""
import numpy as np
import pytest

import oracle
from paper_2511_12051_gb300 import synth


@pytest.mark.parametrize("N,win", [(6, (3, 5, 1, 1)), (9, (5, 11, 3, 6))])
def test_mask_weights_reproduce_the_masked_coherence(N, win):
    H, W = 12, 24
    z = synth.generate(synth.config_spec(4, N=N, H=H, W=W, seed=N)).numpy()
    P, _ = oracle.amp_stats(z)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    C = oracle.covariance(z, win, m)
    Ho, Wo = oracle.out_shape(H, W, win)
    nb = win[0] * win[1]
    for oy in range(Ho):
        for ox in range(Wo):
            s, inside = oracle.window_samples(z, win, oy, ox)
            w = oracle.mask_weights(m[oy, ox], nb)
            assert not np.any(w[~inside])          # the mask never holds samples outside the image
            if cnt[oy, ox] == 0:
                continue
            np.testing.assert_allclose(oracle.weighted_coherence(s, w), C[oy, ox], rtol=1e-12, atol=1e-12)


def test_scale_invariance_and_zero_weights():
    rng = np.random.default_rng(0)
    s = rng.normal(size=(20, 7)) + 1j * rng.normal(size=(20, 7))
    w = rng.uniform(0.2, 2.0, 20)
    C = oracle.weighted_coherence(s, w)
    np.testing.assert_allclose(oracle.weighted_coherence(s, 3.7 * w), C, rtol=1e-13, atol=1e-14)
    w0 = w.copy()
    w0[[3, 11]] = 0.0
    keep = np.ones(20, bool)
    keep[[3, 11]] = False
    np.testing.assert_allclose(oracle.weighted_coherence(s, w0), oracle.weighted_coherence(s[keep], w[keep]),
                               rtol=1e-13, atol=1e-14)


def test_two_samples_by_hand():
    # z(0) = (1, j), z(1) = (2, 2), w = (1, 1/2):  S_00 = 1 + 2 = 3, S_11 = 1 + 2 = 3,
    # S_01 = 1 * conj(j) + (1/2) * 2 * 2 = 2 - j, so C_01 = (2 - j) / 3.
    s = np.array([[1.0, 1j], [2.0, 2.0]])
    C = oracle.weighted_coherence(s, np.array([1.0, 0.5]))
    np.testing.assert_allclose(C, [1.0, (2 - 1j) / 3, 1.0], rtol=0, atol=1e-15)
