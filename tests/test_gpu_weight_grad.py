"""Gradient of L = sum(w * phase) with respect to real per-sample window
weights at the SHP mask (plk_shp_weight_gradient).

- Central finite differences (h = 1e-6) of the FP64 oracle's weighted
  coherence and phase linking over sampled (pixel, window sample) pairs,
  samples inside and outside the mask and border pixels included; three date
  counts (the 8-, 16- and 32-wide register paths), two window geometries.
- Scale invariance of the coherence: per pixel the gradient summed over the
  masked samples is 0.
- On tiling windows (no overlap) each masked sample belongs to one output
  pixel, so dL/dw_b = (1/2) Re(z(q)^H g(q)) with g the gradient of
  plk_phase_link_backward.
- Samples outside the image and pixels without data get 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


@pytest.fixture(scope="module")
def ctx(plk):
    return plk.Context("cuda:0")


def case(N, H, W, win, seed, ref):
    z = synth.generate(synth.config_spec(4, N=N, H=H, W=W, seed=seed)).numpy()
    P, _ = oracle.amp_stats(z)
    m, _ = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    o = oracle.phase_link(oracle.covariance(z, win, m), N, ref)
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1, 1, o["phase"].shape)
    bad = (np.abs(o["phase"]) > np.pi - 0.05).any(axis=0) | (o["status"] == 3) | \
          (o["gap"] < 1e-3 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
    w[:, bad] = 0.0
    return z, m, w.astype(np.float32), bad


def gpu_dw(ctx, z, m, win, ref, w):
    return to_np(ctx.shp_weight_gradient(torch.from_numpy(z).cuda(), win, torch.from_numpy(m.view(np.int64)).cuda(),
                                         ref, torch.from_numpy(w).cuda()))


def pixel_loss(s, weights, N, ref, wp):
    C = oracle.weighted_coherence(s, weights)
    return float(np.dot(wp, oracle.phase_link(C[None], N, ref)["phase"][:, 0]))


@pytest.mark.parametrize("N,win,ref", [(6, (3, 5, 1, 1), 5), (10, (5, 11, 1, 1), 0), (20, (5, 11, 3, 6), 7)])
def test_weight_gradient_matches_oracle_finite_differences(ctx, plk, N, win, ref):
    H, W = 14, 26
    z, m, w, bad = case(N, H, W, win, seed=90 + N, ref=ref)
    dw = gpu_dw(ctx, z, m, win, ref, w)
    Ho, Wo = H // win[2], W // win[3]
    nb = win[0] * win[1]
    assert dw.shape == (Ho, Wo, nb)
    rng = np.random.default_rng(N)
    h = 1e-6
    errs, refs, n_in, n_out = [], [], 0, 0
    # corners, random pixels, and the pixels with the most rejected samples inside the image
    rejected = np.array([[np.sum(oracle.window_samples(z, win, y, x)[1] & (oracle.mask_weights(m[y, x], nb) == 0))
                          for x in range(Wo)] for y in range(Ho)])
    worst = np.argsort(rejected, axis=None)[::-1][:4]
    pix = [(0, 0), (Ho - 1, Wo - 1)] + [(int(rng.integers(Ho)), int(rng.integers(Wo))) for _ in range(4)] + \
        [(int(i // Wo), int(i % Wo)) for i in worst]
    for oy, ox in pix:
        if bad[oy, ox]:
            continue
        s, inside = oracle.window_samples(z.astype(np.complex128), win, oy, ox)
        wts = oracle.mask_weights(m[oy, ox], nb)
        assert np.all(dw[oy, ox, ~inside] == 0.0)
        masked = np.flatnonzero(inside & (wts == 1.0))
        unmasked = np.flatnonzero(inside & (wts == 0.0))
        picks = list(rng.choice(masked, size=min(6, masked.size), replace=False)) + \
            list(rng.choice(unmasked, size=min(4, unmasked.size), replace=False))
        for b in picks:
            wp, wm = wts.copy(), wts.copy()
            wp[b] += h
            wm[b] -= h
            fd = (pixel_loss(s, wp, N, ref, w[:, oy, ox]) - pixel_loss(s, wm, N, ref, w[:, oy, ox])) / (2 * h)
            errs.append(abs(dw[oy, ox, b] - fd))
            refs.append(abs(fd))
            n_in += int(wts[b] == 1.0)
            n_out += int(wts[b] == 0.0)
    errs, refs = np.array(errs), np.array(refs)
    assert n_in > 0 and n_out > 0
    tol = 1e-3 * max(refs.max(), 1e-6) + 5e-3 * refs
    print(f"N={N}: weight gradient vs oracle FD: max abs err {errs.max():.3e}, max |dL/dw| {refs.max():.3e}, "
          f"{n_in} masked and {n_out} unmasked samples")
    assert np.all(errs <= tol), (errs - tol).max()


@pytest.mark.parametrize("N,win", [(8, (5, 11, 1, 1)), (15, (5, 11, 6, 3)), (32, (3, 5, 1, 1))])
def test_masked_weight_gradients_sum_to_zero(ctx, plk, N, win):
    z, m, w, bad = case(N, 24, 40, win, seed=5 + N, ref=1)
    dw = gpu_dw(ctx, z, m, win, 1, w).astype(np.float64)
    nb = win[0] * win[1]
    bits = np.array([[oracle.mask_weights(m[y, x], nb) for x in range(m.shape[1])] for y in range(m.shape[0])])
    tot = (dw * bits).sum(axis=2)
    mag = np.abs(dw * bits).sum(axis=2)
    assert np.all(np.abs(tot) <= 1e-4 * mag + 1e-7), np.max(np.abs(tot) / np.maximum(mag, 1e-30))
    assert np.all(dw[bad] == 0.0)            # zero phase weights give H_p = 0


@pytest.mark.parametrize("N", [9, 24])
def test_weight_gradient_equals_half_re_zg_on_tiling_windows(ctx, plk, N):
    win, ref, H, W = (5, 11, 5, 11), 2, 30, 77
    z, m, w, bad = case(N, H, W, win, seed=30 + N, ref=ref)
    dw = gpu_dw(ctx, z, m, win, ref, w)
    g = to_np(ctx.phase_link_backward(torch.from_numpy(z).cuda(), win, torch.from_numpy(m.view(np.int64)).cuda(),
                                      ref, torch.from_numpy(w).cuda())).astype(np.complex128)
    Ho, Wo = H // 5, W // 11
    q = 0.5 * np.real(np.conj(z.astype(np.complex128)) * g).sum(axis=0)      # [H, W]
    q = q.reshape(Ho, 5, Wo, 11).transpose(0, 2, 1, 3).reshape(Ho, Wo, 55)
    bits = np.array([[oracle.mask_weights(m[y, x], 55) for x in range(Wo)] for y in range(Ho)]).astype(bool)
    scale = np.abs(dw).max()
    np.testing.assert_allclose(dw[bits], q[bits], rtol=2e-3, atol=1e-5 * scale)
    assert np.all(q[~bits] == 0.0)          # unmasked samples carry no gradient on z


def test_no_data_pixels_get_zero(ctx, plk):
    N, win, H, W = 7, (5, 11, 5, 11), 10, 22
    z = synth.generate(synth.config_spec(4, N=N, H=H, W=W, seed=2)).numpy()
    z[:, 0:5, 0:11] = 0
    P, _ = oracle.amp_stats(z)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    assert cnt[0, 0] == 0
    dw = gpu_dw(ctx, z, m, win, 0, np.ones((N, 2, 2), np.float32))
    assert np.all(dw[0, 0] == 0.0)
    assert np.all(np.isfinite(dw))
