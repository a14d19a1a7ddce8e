"""Pins for the oracle's amplitude statistics, GLRT threshold and SHP masks.

Each test ties the oracle to something other than itself: an independent
F-quantile routine, a closed form, exact integer arithmetic, a Monte Carlo
size check, or a mask pattern that is fully determined by construction.
"""
import numpy as np
import pytest

import oracle


def test_glrt_threshold_matches_library_f_quantile():
    stats = pytest.importorskip("scipy.stats")
    for alpha in (1e-3, 1e-2, 0.05):
        for n in (1, 2, 5, 10, 15, 18, 20, 30, 60, 90):
            c = oracle.glrt_threshold(alpha, n)
            ref = stats.f.ppf(1.0 - alpha / 2.0, 2 * n, 2 * n)
            assert abs(c - ref) <= 1e-9 * ref, (alpha, n, c, ref)


def test_glrt_threshold_closed_form_n1():
    # F(2,2) has CDF x/(1+x), so its (1 - a/2) quantile is 2/a - 1.
    for alpha in (1e-3, 0.02, 0.1):
        assert oracle.glrt_threshold(alpha, 1) == pytest.approx(2.0 / alpha - 1.0, rel=1e-12)


def test_glrt_threshold_monotone():
    cs = [oracle.glrt_threshold(1e-3, n) for n in range(1, 40)]
    assert all(a > b for a, b in zip(cs, cs[1:]))
    assert oracle.glrt_threshold(1e-4, 10) > oracle.glrt_threshold(1e-3, 10)


def test_amp_stats_exact_on_integer_samples():
    rng = np.random.default_rng(1)
    n, H, W = 7, 9, 13
    re = rng.integers(-60, 61, size=(n, H, W))
    im = rng.integers(-60, 61, size=(n, H, W))
    z = (re + 1j * im).astype(np.complex64)
    P, A = oracle.amp_stats(z)
    exact = (re.astype(np.int64) ** 2 + im.astype(np.int64) ** 2).sum(0)
    assert np.array_equal(P.astype(np.int64), exact)
    # Pythagorean samples have integer amplitudes: 3+4j -> 5, 5+12j -> 13.
    z2 = np.array([[[3 + 4j]], [[5 + 12j]], [[8 + 15j]]], np.complex64)
    P2, A2 = oracle.amp_stats(z2)
    assert P2[0, 0] == 25 + 169 + 289 and A2[0, 0] == 5 + 13 + 17


def test_amp_stats_accumulate_is_one_float_add():
    rng = np.random.default_rng(2)
    a = (rng.standard_normal((4, 5, 6)) + 1j * rng.standard_normal((4, 5, 6))).astype(np.complex64)
    b = (rng.standard_normal((3, 5, 6)) + 1j * rng.standard_normal((3, 5, 6))).astype(np.complex64)
    Pa, _ = oracle.amp_stats(a)
    Pb, _ = oracle.amp_stats(b)
    Pm, _ = oracle.amp_stats(a)
    oracle.amp_stats(b, Pm, accumulate=True)
    assert np.array_equal(Pm, (Pa + Pb).astype(np.float32))


def _bits(mask_words, nbits):
    out = np.zeros(mask_words.shape[:-1] + (nbits,), bool)
    for b in range(nbits):
        out[..., b] = (mask_words[..., b // 64] >> np.uint64(b % 64)) & np.uint64(1)
    return out


def test_shp_constant_scene_counts_in_image_neighbours():
    H, W, wy, wx = 9, 14, 5, 11
    P = np.full((H, W), 3.5, np.float32)
    mask, count = oracle.shp_select(P, (wy, wx, 1, 1), np.float32(2.0))
    for i in range(H):
        for j in range(W):
            ny = min(H - 1, i + 2) - max(0, i - 2) + 1
            nx = min(W - 1, j + 5) - max(0, j - 5) + 1
            assert count[i, j] == ny * nx


def test_shp_checkerboard_pattern():
    H, W, wy, wx = 12, 20, 5, 11
    yy, xx = np.mgrid[0:H, 0:W]
    P = np.where((yy + xx) % 2 == 0, 1.0, 100.0).astype(np.float32)
    c = oracle.glrt_threshold(1e-3, 10)  # ~4.75, far below the ratio 100
    mask, count = oracle.shp_select(P, (wy, wx, 1, 1), np.float32(c))
    bits = _bits(mask, wy * wx)
    for i in range(H):
        for j in range(W):
            for dy in range(-2, 3):
                for dx in range(-5, 6):
                    y, x = i + dy, j + dx
                    inside = 0 <= y < H and 0 <= x < W
                    want = inside and (dy + dx) % 2 == 0
                    assert bits[i, j, (dy + 2) * wx + dx + 5] == want


def test_shp_symmetric_at_stride_one():
    rng = np.random.default_rng(3)
    H, W, wy, wx = 24, 30, 5, 11
    P = rng.gamma(10.0, 1.0, size=(H, W)).astype(np.float32)
    mask, _ = oracle.shp_select(P, (wy, wx, 1, 1), np.float32(1.6))
    bits = _bits(mask, wy * wx)
    for i in range(H):
        for j in range(W):
            for dy in range(-2, 3):
                for dx in range(-5, 6):
                    y, x = i + dy, j + dx
                    if 0 <= y < H and 0 <= x < W:
                        b1 = bits[i, j, (dy + 2) * wx + dx + 5]
                        b2 = bits[y, x, (-dy + 2) * wx + (-dx) + 5]
                        assert b1 == b2


def test_shp_threshold_edge_is_inclusive_and_float():
    # ratio exactly c is accepted; the next float above c is rejected.
    c = np.float32(3.0)
    up = np.nextafter(np.float32(3.0), np.float32(4.0))
    P = np.array([[1.0, 3.0]], np.float32)
    bits = _bits(oracle.shp_select(P, (1, 3, 1, 1), c)[0], 3)
    assert bits[0, 0].tolist() == [False, True, True]   # 3 <= 3 * 1: accepted
    assert bits[0, 1].tolist() == [True, True, False]
    P = np.array([[1.0, up]], np.float32)
    bits = _bits(oracle.shp_select(P, (1, 3, 1, 1), c)[0], 3)
    assert bits[0, 0].tolist() == [False, True, False]  # 3+ulp > 3 * 1: rejected
    assert bits[0, 1].tolist() == [False, True, False]


def test_shp_no_data_pixels():
    P = np.ones((5, 5), np.float32)
    P[2, 2] = 0.0
    P[0, 0] = 0.0
    mask, count = oracle.shp_select(P, (3, 3, 1, 1), np.float32(2.0))
    assert count[2, 2] == 0 and not mask[2, 2].any()
    assert count[1, 1] == 7  # 9 minus the two zero-power pixels (0,0), (2,2)


def test_shp_output_grid_centres():
    # Spikes at the decimation-window centres; with a window narrower than the
    # stride only the centre itself is homogeneous with a spiked centre.
    H, W, sy, sx = 17, 40, 3, 6
    P = np.ones((H, W), np.float32)
    Ho, Wo = H // sy, W // sx
    for i in range(Ho):
        for j in range(Wo):
            P[i * sy + sy // 2, j * sx + sx // 2] = 1e6
    mask, count = oracle.shp_select(P, (3, 5, sy, sx), np.float32(4.0))
    assert mask.shape[:2] == (Ho, Wo)
    assert np.all(count == 1)
    bits = _bits(mask, 15)
    assert np.all(bits[..., 7])  # the centre bit (1*5 + 2)


def test_glrt_size_on_homogeneous_rayleigh_scene():
    # Under equal scale each (centre, neighbour) pair is rejected with
    # probability alpha exactly; check the empirical rate.
    rng = np.random.default_rng(4)
    n, H, W = 10, 260, 260
    z = ((rng.standard_normal((n, H, W)) + 1j * rng.standard_normal((n, H, W))) / np.sqrt(2)).astype(np.complex64)
    P, _ = oracle.amp_stats(z)
    alpha = 0.05
    c = oracle.glrt_threshold(alpha, n)
    mask, count = oracle.shp_select(P, (3, 3, 1, 1), np.float32(c))
    inner = count[1:-1, 1:-1].astype(np.float64)
    pairs = inner.size * 8
    rejected = pairs - (inner.sum() - inner.size)
    rate = rejected / pairs
    sd = np.sqrt(alpha * (1 - alpha) / pairs) * 3.0  # pairs share centres: inflate
    assert abs(rate - alpha) < 5 * sd, (rate, alpha, sd)
