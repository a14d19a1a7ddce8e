"""Pins for the oracle's phase cosine similarity gamma_s (Sec. III-C,
eq. (phase-cosine-sim)).

* Fields whose interferograms agree everywhere (one phase history plus a
  constant offset per pixel) give gamma_s = 1.
* An island pixel whose history differs by a ramp delta*t has every
  similarity equal to the closed form
  c = [(M-1) cos d + (M-2) cos 2d + (M-3) cos 3d] / (3M - 6), so gamma_s = c.
* A pi shift on one date j changes the sign of the cosines of exactly the
  network pairs containing j: s = (N_ifg - 2 n_j) / N_ifg with n_j = 3 at the
  first/last date, 6 inside; this pins the nearest-3 network.
* Radius 1 (the 4-neighbour disk, not the 8-neighbour square) with two equal
  and two unequal neighbours: the even-count median (1 + c) / 2; the square
  would give c.
* Invariances: a per-date phase common to all pixels, and adding 2 pi.
* Independent uniform phases: gamma_s near the population median of the
  similarity, drawn by Monte Carlo (slightly negative: the sum is skewed).
* Missing data: NaN centres, NaN neighbours left out, image edges.
* Brute force with plain Python loops on tiny inputs.
"""
import math
import statistics

import numpy as np
import pytest

import oracle


def closed_form(delta, M):
    ds = [d for d in (1, 2, 3) if d < M]
    K = sum(M - d for d in ds)
    return sum((M - d) * math.cos(d * delta) for d in ds) / K


def base_field(M, Ho, Wo, seed):
    rng = np.random.default_rng(seed)
    hist = np.cumsum(rng.normal(0, 0.5, M))                   # one phase history for all pixels
    psi = rng.uniform(-np.pi, np.pi, (Ho, Wo))                # a constant offset per pixel
    return hist[:, None, None] + psi[None]


def test_network_and_window_sizes():
    assert len(oracle.nearest3_pairs(15)) == 39 == 3 * 15 - 6
    assert len(oracle.nearest3_pairs(3)) == 3 and len(oracle.nearest3_pairs(2)) == 1
    assert set(oracle.nearest3_pairs(5)) == {(0, 1), (1, 2), (2, 3), (3, 4), (0, 2), (1, 3), (2, 4), (0, 3), (1, 4)}
    # lattice points of the disk, centre excluded (Gauss circle counts)
    assert [len(oracle.disk_offsets(r)) for r in (1, 2, 3, 7)] == [4, 12, 28, 148]


def test_agreeing_interferograms_give_one():
    g = oracle.phase_similarity(base_field(15, 20, 24, 0), 4)
    np.testing.assert_allclose(g, 1.0, atol=1e-12)


@pytest.mark.parametrize("M,delta", [(15, 0.3), (6, 1.1), (3, 2.0), (2, 0.7)])
def test_island_closed_form(M, delta):
    ph = base_field(M, 15, 17, 1)
    t = np.arange(M)
    ph[:, 7, 8] += delta * t
    g = oracle.phase_similarity(ph, 3)
    assert abs(g[7, 8] - closed_form(delta, M)) < 1e-12
    # its neighbours see it once among 28: their median stays 1
    assert abs(g[7, 9] - 1.0) < 1e-12 and abs(g[5, 8] - 1.0) < 1e-12


@pytest.mark.parametrize("j,n_j", [(0, 3), (1, 4), (2, 5), (7, 6), (13, 4), (14, 3)])
def test_pi_shift_on_one_date_pins_the_network(j, n_j):
    M = 15
    K = 3 * M - 6
    ph = base_field(M, 13, 13, 2)
    ph[j, 6, 6] += np.pi
    g = oracle.phase_similarity(ph, 2)
    assert abs(g[6, 6] - (K - 2 * n_j) / K) < 1e-12


def test_radius_one_is_the_four_neighbour_disk_and_even_median():
    M, delta = 8, 0.9
    ph = base_field(M, 3, 3, 3)
    t = np.arange(M)
    for (y, x) in [(0, 1), (1, 2), (0, 0), (0, 2), (2, 0), (2, 2)]:   # two edge and four corner pixels differ
        ph[:, y, x] += delta * t
    g = oracle.phase_similarity(ph, 1)
    c = closed_form(delta, M)
    assert abs(g[1, 1] - (1.0 + c) / 2) < 1e-12              # the 8-neighbour square would give c


def test_invariances():
    rng = np.random.default_rng(4)
    ph = rng.uniform(-np.pi, np.pi, (10, 16, 18))
    g = oracle.phase_similarity(ph, 3)
    common = rng.uniform(-5, 5, 10)[:, None, None]             # atmosphere-like, the same at every pixel
    np.testing.assert_allclose(oracle.phase_similarity(ph + common, 3), g, atol=1e-12)
    wraps = 2 * np.pi * rng.integers(-3, 4, ph.shape)
    np.testing.assert_allclose(oracle.phase_similarity(ph + wraps, 3), g, atol=1e-12)
    assert np.all(g <= 1.0 + 1e-15)


def test_independent_phases_match_the_population_median():
    # For independent uniform phases each similarity is the mean of cos(t_b - t_a)
    # over the network with t iid uniform: zero mean but skewed (for a full
    # network the sum is (|sum e^{jt}|^2 - M) / 2), so its median is slightly
    # negative.  Per-pixel medians over the window must sit near the population
    # median, drawn here by Monte Carlo straight from that distribution.
    rng = np.random.default_rng(5)
    M = 15
    g = oracle.phase_similarity(rng.uniform(-np.pi, np.pi, (M, 60, 60)), 5)
    th = rng.uniform(-np.pi, np.pi, (200000, M))
    terms = [np.cos(th[:, a + d] - th[:, a]) for d in (1, 2, 3) for a in range(M - d)]
    m_pop = float(np.median(np.mean(terms, axis=0)))
    assert -0.02 < m_pop < -0.005
    assert abs(float(np.mean(g)) - m_pop) < 0.003 and float(np.std(g)) < 0.05


def test_missing_data_and_edges():
    M = 6
    ph = base_field(M, 9, 10, 6)
    t = np.arange(M)
    ph[:, 0, 0] += 0.5 * t
    ph[2, 4, 4] = np.nan                                      # a no-data cell
    g = oracle.phase_similarity(ph, 1)
    assert np.isnan(g[4, 4])
    # (4, 5) has neighbours (3,5), (5,5), (4,6) and the no-data (4,4): three left, all equal
    assert abs(g[4, 5] - 1.0) < 1e-12
    # the corner (0, 0) has two neighbours, both with the closed-form similarity
    assert abs(g[0, 0] - closed_form(0.5, M)) < 1e-12
    # a pixel whose every neighbour is no-data
    ph2 = base_field(M, 3, 3, 7)
    ph2[0, 0, 1] = ph2[0, 1, 0] = ph2[0, 1, 2] = ph2[0, 2, 1] = np.nan
    assert np.isnan(oracle.phase_similarity(ph2, 1)[1, 1])


def brute_force(ph, r):
    """Plain loops: per pixel, per disk neighbour, per nearest-3 pair."""
    M, Ho, Wo = ph.shape
    out = np.full((Ho, Wo), np.nan)
    for y in range(Ho):
        for x in range(Wo):
            if not all(math.isfinite(ph[i, y, x]) for i in range(M)):
                continue
            sims = []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    if (dy, dx) == (0, 0) or dy * dy + dx * dx > r * r:
                        continue
                    yy, xx = y + dy, x + dx
                    if not (0 <= yy < Ho and 0 <= xx < Wo):
                        continue
                    if not all(math.isfinite(ph[i, yy, xx]) for i in range(M)):
                        continue
                    terms = []
                    for d in (1, 2, 3):
                        for a in range(M - d):
                            b = a + d
                            terms.append(math.cos((ph[b, y, x] - ph[a, y, x]) - (ph[b, yy, xx] - ph[a, yy, xx])))
                    sims.append(sum(terms) / len(terms))
            if sims:
                out[y, x] = statistics.median(sims)
    return out


@pytest.mark.parametrize("M,r", [(5, 2), (9, 3), (2, 1), (4, 4)])
def test_brute_force_tiny(M, r):
    rng = np.random.default_rng(M * 10 + r)
    ph = rng.uniform(-np.pi, np.pi, (M, 7, 9))
    ph[:, 3, 4] = np.nan
    np.testing.assert_allclose(oracle.phase_similarity(ph, r), brute_force(ph, r), atol=1e-12, equal_nan=True)
