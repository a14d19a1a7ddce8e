"""Pins for the oracle's persistent-scatterer selection and regridding
(Sec. III-A, D_A = sigma_A / mu_A; Sec. IV, PS threshold; Supplement,
"Regridding PS and DS to 30 m resolution").

* D_A: exact values on amplitude sequences whose mean and population
  deviation are exact in binary; the Rayleigh closed form sqrt(4/pi - 1) on
  fully developed speckle; numpy's mean / std of |z| in double on random
  stacks; the pooled statistics of two groups by eqs. (merged-mean),
  (merged-variance) against sums merged over the same two groups.
* Regridding: the three cases of the Supplement on planted scatterers (none,
  one, several with different D_A in either position order), ties to the
  first in row-major order, the threshold boundary, the blocks that take the
  rows and columns beyond the grid, pixels with no amplitude or a zero sample.
* PS compression: kappa = (sum_i |z_i|) times the unit phasor of z_ref
  (z_shift when re-referenced), a closed form of the definition.
* Chain: a planted PS with its own phase history, inside a DS background,
  keeps the day-1 datum across mini-stacks in both reference schemes.
"""
import numpy as np
import pytest

import oracle
from paper_2511_12051_gb300 import synth

RAYLEIGH_DA = np.sqrt(4.0 / np.pi - 1.0)  # sigma / mu of a Rayleigh law


def sums(amps, phases=None):
    amps = np.asarray(amps, np.float32)
    z = amps.astype(np.complex64) if phases is None else (amps * np.exp(1j * phases)).astype(np.complex64)
    return oracle.amp_stats(z)


def test_amp_dispersion_exact_values():
    n = 8
    a = np.ones((n, 1, 4), np.float32)
    a[:, 0, 0] = 2.0                          # constant -> 0
    a[:, 0, 1] = [1, 3] * 4                   # mu 2, sigma 1 -> 0.5
    a[:, 0, 2] = [3, 5] * 4                   # mu 4, sigma 1 -> 0.25
    a[:, 0, 3] = [0, 0, 0, 0, 0, 0, 0, 0]     # no amplitude -> NaN
    sp, sa = sums(a)
    da = oracle.amp_dispersion(sp, sa, n)
    assert da[0, 0] == 0.0 and da[0, 1] == 0.5 and da[0, 2] == 0.25
    assert np.isnan(da[0, 3])


def test_amp_dispersion_rayleigh_closed_form():
    rng = np.random.default_rng(0)
    n, H, W = 400, 16, 16
    z = ((rng.standard_normal((n, H, W)) + 1j * rng.standard_normal((n, H, W))) / np.sqrt(2)).astype(np.complex64)
    sp, sa = oracle.amp_stats(z)
    da = oracle.amp_dispersion(sp, sa, n)
    # the mean over 256 pixels of 400 samples each: standard error ~ 1e-3
    assert abs(float(np.mean(da)) - RAYLEIGH_DA) < 5e-3
    # speckle is far from any PS threshold of practice
    assert np.all(da > 0.35)


def test_amp_dispersion_matches_numpy_statistics():
    rng = np.random.default_rng(1)
    n, H, W = 25, 20, 30
    amp = rng.uniform(0.5, 2.0, (H, W))[None] * rng.gamma(20.0, 1 / 20.0, (n, H, W))
    z = (amp * np.exp(1j * rng.uniform(-np.pi, np.pi, (n, H, W)))).astype(np.complex64)
    sp, sa = oracle.amp_stats(z)
    da = oracle.amp_dispersion(sp, sa, n)
    A = np.abs(z.astype(np.complex128))
    want = A.std(axis=0) / A.mean(axis=0)
    # single-precision sums and the cancellation in E[A^2] - mu^2
    np.testing.assert_allclose(da, want, rtol=2e-4)


def test_amp_dispersion_merged_groups():
    # two groups of images with their own mean and variance, pooled with
    # weights n_1, n_2 by eqs. (merged-mean), (merged-variance)
    rng = np.random.default_rng(2)
    H, W, n1, n2 = 6, 7, 10, 15
    z1 = (rng.gamma(9, 1 / 9, (n1, H, W)) * np.exp(1j * rng.uniform(0, 6, (n1, H, W)))).astype(np.complex64)
    z2 = (1.5 * rng.gamma(9, 1 / 9, (n2, H, W)) * np.exp(1j * rng.uniform(0, 6, (n2, H, W)))).astype(np.complex64)
    sp, sa = oracle.amp_stats(z1)
    oracle.amp_stats(z2, sp, sa, accumulate=True)
    da = oracle.amp_dispersion(sp, sa, n1 + n2)
    A1, A2 = np.abs(z1.astype(np.complex128)), np.abs(z2.astype(np.complex128))
    mu = (n1 * A1.mean(0) + n2 * A2.mean(0)) / (n1 + n2)
    var = (n1 * (A1.var(0) + A1.mean(0) ** 2) + n2 * (A2.var(0) + A2.mean(0) ** 2)) / (n1 + n2) - mu ** 2
    np.testing.assert_allclose(da, np.sqrt(var) / mu, rtol=2e-4)


# ------------------------------------------------------------------ regrid

def background(N, H, W, seed):
    """DS background whose amplitudes alternate between 0.2 a and 1.8 a (in a
    random order per pixel): D_A near 0.8 for any even N, never a PS at the
    thresholds below 0.6 used here; random phases."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 2.0, (H, W))
    lo = rng.integers(0, 2, (H, W))
    alt = np.where((np.arange(N)[:, None, None] + lo[None]) % 2 == 0, 0.2, 1.8) * a[None]
    return (alt * np.exp(1j * rng.uniform(-np.pi, np.pi, (N, H, W)))).astype(np.complex64)


def plant(z, y, x, amps, phases):
    z[:, y, x] = (np.asarray(amps, np.float64) * np.exp(1j * np.asarray(phases))).astype(np.complex64)


def regrid(z, window, da_max, first_real=0, ref=0, ds_phase=None, ds_status=None):
    N, H, W = z.shape
    Ho, Wo = H // window[2], W // window[3]
    sp, sa = oracle.amp_stats(z[first_real:])
    if ds_phase is None:
        ds_phase = np.full((N - first_real, Ho, Wo), 7.0)     # a marker no phase takes
    if ds_status is None:
        ds_status = np.zeros((Ho, Wo), np.uint8)
    return oracle.ps_regrid(z, first_real, window, sp, sa, N - first_real, ref, da_max, ds_phase, ds_status)


def test_regrid_three_cases():
    N, H, W, win = 12, 9, 24, (3, 7, 3, 6)               # 3 x 4 cells of 3 x 6 pixels
    z = background(N, H, W, 3)
    t = np.arange(N)
    hist_a = 0.7 * t + 0.3 * np.sin(2 * t)                 # PS a: constant amplitude, D_A = 0
    hist_b = -0.4 * t                                      # PS b: amplitudes 1, 1.2: D_A = 1/11
    plant(z, 1, 8, 2.0, hist_a)                            # cell (0, 1): one PS
    plant(z, 4, 2, 2.0, hist_a + 1.0)                      # cell (1, 0): a and b, a first in row-major order
    plant(z, 5, 4, [1.0, 1.2] * 6, hist_b)
    plant(z, 7, 13, [1.0, 1.2] * 6, hist_b)                # cell (2, 2): b first, a second
    plant(z, 8, 16, 3.0, hist_a)
    ph, st = regrid(z, win, 0.2)
    want = np.angle(np.exp(1j * (hist_a - hist_a[0])))
    np.testing.assert_allclose(ph[:, 0, 1], want, atol=1e-6, rtol=0)
    np.testing.assert_allclose(ph[:, 1, 0], want, atol=1e-6, rtol=0)     # lowest D_A: a
    np.testing.assert_allclose(ph[:, 2, 2], want, atol=1e-6, rtol=0)     # lowest D_A: a, in the other order
    assert st[0, 1] == st[1, 0] == st[2, 2] == oracle.PS_STATUS
    # every other cell keeps its DS phases and status
    keep = np.ones((3, 4), bool)
    keep[0, 1] = keep[1, 0] = keep[2, 2] = False
    assert np.all(ph[:, keep] == 7.0) and np.all(st[keep] == 0)
    # the reference date's PS phase is exactly zero
    assert np.all(ph[0, ~keep] == 0.0)
    # with b alone eligible (threshold between the two) cell (2, 2) takes b
    z2 = z.copy()
    plant(z2, 8, 16, [1.0, 4.0] * 6, hist_a)               # a's D_A now 0.6
    ph2, st2 = regrid(z2, win, 0.2)
    np.testing.assert_allclose(ph2[:, 2, 2], np.angle(np.exp(1j * (hist_b - hist_b[0]))), atol=1e-6, rtol=0)


def test_regrid_tie_goes_to_first_in_row_major_order():
    N, win = 10, (3, 5, 3, 6)
    z = background(N, 6, 12, 4)
    t = np.arange(N)
    plant(z, 2, 1, 1.5, 0.5 * t)       # row 2
    plant(z, 1, 4, 2.5, -0.5 * t)      # row 1: first in row-major order, same D_A = 0
    ph, st = regrid(z, win, 0.1)
    np.testing.assert_allclose(ph[:, 0, 0], np.angle(np.exp(-0.5j * t)), atol=1e-6, rtol=0)


def test_regrid_threshold_boundary():
    N, win = 8, (3, 5, 3, 6)
    z = background(N, 3, 6, 5)
    plant(z, 1, 1, [1.0, 3.0] * 4, np.zeros(N))            # real samples: D_A = 0.5 exactly
    _, st = regrid(z, win, 0.5)
    assert st[0, 0] == oracle.PS_STATUS
    _, st = regrid(z, win, np.nextafter(np.float32(0.5), np.float32(0)))
    assert st[0, 0] == 0


def test_regrid_leftover_rows_and_columns():
    # H = 11, W = 27 with 3 x 6 cells: Ho = 3, Wo = 4; rows 9-10 and columns
    # 24-26 belong to the last cell row and column.
    N, win = 9, (3, 5, 3, 6)
    z = background(N, 11, 27, 6)
    t = np.arange(N)
    plant(z, 10, 26, 1.0, 0.3 * t)
    plant(z, 10, 2, 1.0, -0.3 * t)
    ph, st = regrid(z, win, 0.2)
    assert st[2, 3] == oracle.PS_STATUS and st[2, 0] == oracle.PS_STATUS
    np.testing.assert_allclose(ph[:, 2, 3], np.angle(np.exp(0.3j * t)), atol=1e-6, rtol=0)
    np.testing.assert_allclose(ph[:, 2, 0], np.angle(np.exp(-0.3j * t)), atol=1e-6, rtol=0)
    assert np.sum(st == oracle.PS_STATUS) == 2


def test_regrid_degenerate_pixels_never_ps():
    # With a threshold above every dispersion each block takes its lowest-D_A
    # pixel, except a pixel with no amplitude (D_A undefined) or with a zero
    # sample (its phase on that date undefined), even where its D_A is lowest.
    N, win = 6, (3, 5, 3, 6)
    z = background(N, 3, 12, 7)
    z[:, 0, 0] = 0                                         # cell (0, 0): no amplitude
    plant(z, 1, 8, 1.0, np.zeros(N))                       # cell (0, 1): D_A would be 0.447 ...
    z[3, 1, 8] = 0                                         # ... but one sample is zero
    sp, sa = oracle.amp_stats(z)
    da = oracle.amp_dispersion(sp, sa, N)
    assert np.isnan(da[0, 0]) and da[1, 8] == np.nanmin(da[:, 6:])
    ph, st = regrid(z, win, 1e6)
    assert np.all(st == oracle.PS_STATUS)
    for cj, skip in ((0, (0, 0)), (1, (1, 2))):
        d = da[:, 6 * cj:6 * cj + 6].astype(np.float64)
        d[skip] = np.inf
        y, x = np.unravel_index(int(np.argmin(d)), d.shape)
        zq = z[:, y, 6 * cj + x].astype(np.complex128)
        np.testing.assert_allclose(ph[:, 0, cj], np.angle(zq * np.conj(zq[0])), rtol=0, atol=1e-12)


def test_regrid_phases_relative_to_a_compressed_reference():
    # reference entry 0 is a compressed SLC, real dates 1..N-1
    N, win = 7, (3, 5, 3, 6)
    z = background(N, 3, 6, 8)
    t = np.arange(1, N)
    plant(z[1:], 2, 3, 1.0, 0.4 * t)
    z[0, 2, 3] = np.complex64(np.exp(0.25j))               # kappa carries phase 0.25
    ph, st = regrid(z, win, 0.2, first_real=1, ref=0)
    assert ph.shape == (N - 1, 1, 1) and st[0, 0] == oracle.PS_STATUS
    np.testing.assert_allclose(ph[:, 0, 0], np.angle(np.exp(1j * (0.4 * t - 0.25))), atol=1e-6)


# --------------------------------------------------------------- compress

@pytest.mark.parametrize("shift", [-1, 5])
def test_ps_compress_closed_form(shift):
    N, H, W, first_real, ref = 6, 5, 7, 1, 0
    rng = np.random.default_rng(9)
    z = background(N, H, W, 9).astype(np.complex128)
    sp, sa = oracle.amp_stats(z[first_real:].astype(np.complex64))
    base = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    k = oracle.ps_compress(z, first_real, sp, sa, N - first_real, ref, 1e6, base, shift=shift)
    anchor = z[shift] if shift >= 0 else z[ref]
    want = np.abs(z[first_real:]).sum(0) * anchor / np.abs(anchor)
    np.testing.assert_allclose(k, want, rtol=1e-12, atol=1e-12)
    # below every pixel's dispersion nothing changes
    k0 = oracle.ps_compress(z, first_real, sp, sa, N - first_real, ref, 1e-3, base, shift=shift)
    assert np.array_equal(k0, base)


# ------------------------------------------------------------------ chain

@pytest.mark.parametrize("scheme", ["first", "last"])
def test_chain_ps_keeps_its_datum(scheme):
    # A PS whose phase history differs from the DS background: its cell must
    # report the PS's history relative to the datum of the scheme in every
    # mini-stack, which needs kappa formed on the PS's own phases.
    n_dates, M, H, W, win = 20, 5, 12, 24, (3, 5, 3, 6)
    t = np.arange(n_dates)
    phi_ds = 0.2 * t
    phi_ps = 0.9 * t + 0.5 * np.sin(t)
    rng = np.random.default_rng(10)
    psi = rng.uniform(-np.pi, np.pi, (H, W))
    # background amplitudes of the fixture above (D_A near 0.8), DS phase history
    amp = np.abs(background(n_dates, H, W, 10)).astype(np.float64)
    z = (amp * np.exp(1j * (phi_ds[:, None, None] + psi[None]))).astype(np.complex64)
    plant(z, 4, 9, 3.0, phi_ps + 1.3)                      # cell (1, 1)
    ch = oracle.OracleChain(H, W, win, K_max=3, alpha=1e-3, scheme=scheme, ps_da_max=0.2)
    for s, sl in enumerate(synth.ministack_slices(n_dates, M)):
        out = ch.step(z[sl])
        assert out["status"][1, 1] == oracle.PS_STATUS
        assert np.sum(out["status"] == oracle.PS_STATUS) == 1
        ref_date = 0 if (s == 0 or scheme == "first") else sl.start - 1
        want = np.angle(np.exp(1j * (phi_ps[sl] - phi_ps[ref_date])))
        np.testing.assert_allclose(np.angle(np.exp(1j * (out["phase_real"][:, 1, 1] - want))), 0, atol=1e-5)


def test_regrid_lowest_da_without_reference_sample_gives_way():
    # The lowest-D_A pixel of the block has a zero reference sample (a
    # compressed SLC that was zero there): the next lowest is taken.
    N, win = 9, (3, 5, 3, 6)
    z = background(N, 3, 6, 11)
    t = np.arange(1, N)
    plant(z[1:], 0, 4, 2.0, 0.1 * t)                       # D_A = 0, but ...
    z[0, 0, 4] = 0                                         # ... no reference sample
    plant(z[1:], 2, 1, [1.0, 1.2] * 4, -0.2 * t)           # D_A = 1/11
    z[0, 2, 1] = np.complex64(1.0)
    ph, st = regrid(z, win, 0.2, first_real=1, ref=0)
    assert st[0, 0] == oracle.PS_STATUS
    np.testing.assert_allclose(ph[:, 0, 0], np.angle(np.exp(-0.2j * t)), atol=1e-6, rtol=0)
