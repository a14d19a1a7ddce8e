"""Pins for the oracle's mini-stack chain (Sec. II-B) and estimator quality.

* Noise-free stacks: the chain must return the true phase history relative to
  the first date of the archive, exactly, across mini-stacks (the always-first
  compressed-SLC reference of Fig. 1 needs no datum adjustment).
* A phase step on a patch appears, relative to day 1, in every later
  mini-stack.
* Statistical: on exponential-decay stacks with a known phase ramp the RMS
  wrapped error falls as the number of looks grows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth


def wrapped(a):
    return np.angle(np.exp(1j * a))


def noise_free_stack(n_dates, H, W, seed=0):
    rng = np.random.default_rng(seed)
    t = np.arange(n_dates)
    phi = 0.3 * t + 0.4 * np.sin(t)          # nonlinear history, wraps several times
    amp = rng.rayleigh(1.0, (H, W)) + 0.2
    psi = rng.uniform(-np.pi, np.pi, (H, W))  # scatterer phase, constant in time
    z = amp[None] * np.exp(1j * (phi[:, None, None] + psi[None]))
    return z.astype(np.complex64), phi


@pytest.mark.parametrize("window", [(3, 5, 1, 1), (5, 11, 3, 6)])
def test_chain_noise_free_returns_truth_relative_to_day_one(window):
    n_dates, M, H, W = 20, 5, 18, 36
    z, phi = noise_free_stack(n_dates, H, W)
    ch = oracle.OracleChain(H, W, window, K_max=3, alpha=1e-3)
    Ho, Wo = H // window[2], W // window[3]
    for s, sl in enumerate(synth.ministack_slices(n_dates, M)):
        out = ch.step(z[sl])
        assert out["K_used"] == min(s, 3)
        got = out["phase_real"]
        want = (phi[sl] - phi[0])[:, None, None]
        assert got.shape == (M, Ho, Wo)
        np.testing.assert_allclose(wrapped(got - want), 0, atol=1e-6)
    assert len(ch.ring) == 3 and ch.n == n_dates


def test_chain_reference_is_newest_compressed_slc():
    # Step 2 of a noise-free chain: the linked phase of the reference entry
    # (the one kappa) is zero and the real dates are relative to day 1.
    n_dates, M, H, W = 10, 5, 9, 15
    z, phi = noise_free_stack(n_dates, H, W, seed=1)
    ch = oracle.OracleChain(H, W, (3, 5, 1, 1), K_max=6)
    ch.step(z[:5])
    out = ch.step(z[5:])
    assert out["N"] == 6 and out["K_used"] == 1
    assert np.all(out["phase"][0] == 0.0)
    np.testing.assert_allclose(wrapped(out["phase_real"] - (phi[5:] - phi[0])[:, None, None]), 0, atol=1e-6)


def test_chain_carries_phase_step_across_ministacks():
    # 20 dates in mini-stacks of 5; +2 rad from date 11 (index 10) on a patch.
    H, W = 48, 96
    spec = synth.StackSpec(N=20, H=H, W=W, rho0=0.9, rho_inf=0.5, tau=60.0, ramp=0.05,
                           step=(10, 12, 36, 30, 66, 2.0), seed=11)
    z = synth.generate(spec).numpy()
    truth = synth.true_phase(spec).numpy()
    ch = oracle.OracleChain(H, W, (5, 11, 1, 1), K_max=3, alpha=1e-3)
    for sl in synth.ministack_slices(20, 5):
        out = ch.step(z[sl])
        err = wrapped(out["phase_real"] - (truth[sl] - truth[0]))
        inner = err[:, 16:32, 36:60]          # patch interior, > half-window from its edge
        outer = err[:, 2:10, 5:25]
        assert np.abs(np.median(inner, axis=(1, 2))).max() < 0.1
        assert np.abs(np.median(outer, axis=(1, 2))).max() < 0.1


def test_rms_error_decreases_with_looks():
    N, H, W = 10, 64, 64
    errs = []
    windows = [(1, 3, 1, 1), (3, 5, 1, 1), (5, 11, 1, 1), (11, 21, 1, 1)]
    for window in windows:
        e = []
        for seed in range(4):
            spec = synth.config_spec(0, H=H, W=W, seed=100 + seed)
            z = synth.generate(spec).numpy()
            truth = synth.true_phase(spec).numpy()
            P = np.ones((H, W), np.float32)  # accept every neighbour
            mask, _ = oracle.shp_select(P, window, np.float32(2.0))
            C = oracle.covariance(z, window, mask)
            out = oracle.phase_link(C.reshape(-1, N * (N + 1) // 2), N, ref=0)
            ph = out["phase"].reshape(N, H, W)
            hy, hx = window[0] // 2, window[1] // 2
            d = wrapped(ph - (truth - truth[0]))[1:, hy:H - hy, hx:W - hx]
            e.append(np.sqrt(np.mean(d ** 2)))
        errs.append(np.mean(e))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.25 * errs[0], errs


@pytest.mark.parametrize("window", [(3, 5, 1, 1), (5, 11, 3, 6)])
def test_chain_last_real_scheme_noise_free(window):
    # Production scheme (Sec. IV; Supplement): each compressed SLC carries the
    # phase of its mini-stack's last real date, so the outputs of step s are
    # the short-baseline interferograms to the last date of step s-1 (to day 1
    # on the first step), exactly on noise-free stacks.
    n_dates, M, H, W = 20, 5, 18, 36
    z, phi = noise_free_stack(n_dates, H, W, seed=2)
    ch = oracle.OracleChain(H, W, window, K_max=3, alpha=1e-3, scheme="last")
    for s, sl in enumerate(synth.ministack_slices(n_dates, M)):
        out = ch.step(z[sl])
        ref_date = 0 if s == 0 else sl.start - 1
        want = (phi[sl] - phi[ref_date])[:, None, None]
        np.testing.assert_allclose(wrapped(out["phase_real"] - want), 0, atol=1e-6)
        assert np.all(out["phase"][out["K_used"] - 1] == 0.0) if out["K_used"] else True


def test_chain_last_real_kappa_is_rotated_first_kappa():
    # The last-real compressed SLC is the always-first one rotated, cell by
    # cell, by the linked phase of the last real date: kappa_last =
    # kappa_first * exp(j phase_last(cell)).
    spec = synth.config_spec(0, N=8, H=24, W=36, seed=5)
    z = synth.generate(spec).numpy()
    window = (5, 11, 3, 6)
    a = oracle.OracleChain(24, 36, window, K_max=2, scheme="first")
    b = oracle.OracleChain(24, 36, window, K_max=2, scheme="last")
    oa, ob = a.step(z), b.step(z)
    np.testing.assert_allclose(oa["phase"], ob["phase"])  # same linking on the first step
    last = oa["phase"][-1]
    Ho, Wo = last.shape
    ci = np.minimum(np.arange(24) // 3, Ho - 1)
    cj = np.minimum(np.arange(36) // 6, Wo - 1)
    rot = np.exp(1j * last[ci[:, None], cj[None, :]])
    ok = np.isfinite(rot)
    np.testing.assert_allclose(b.ring[-1][ok], (a.ring[-1] * rot)[ok], rtol=1e-12, atol=1e-9)
