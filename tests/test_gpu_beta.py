"""The regularised EMI (Sec. III-B: G = (1 - beta)|C| + beta I) on the GPU,
beta > 0, against the FP64 oracle:

- phase linking on coherences of the 128x128 and burst-shaped workloads:
  phase within 1e-4 rad, gamma_t within 1e-5, no-data pixels alike; also
  without regularisation for a caller's shift below or above lambda_min;
- the adjoint: central finite differences of the oracle (h = 1e-6) on sampled
  samples (its (1 - beta) term of the G^-1 derivative is otherwise not
  exercised);
- phase uncertainty and the window-weight gradient against the oracle's
  finite differences on small cases.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import clear_of_degenerate, PHASE_TOL, TCOH_TOL, phase_report, to_np

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


def case(cfg, N, H, W, win, seed):
    z = synth.generate(synth.config_spec(cfg, N=N, H=H, W=W, seed=seed)).numpy()
    P, _ = oracle.amp_stats(z)
    m, _ = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    return z, m


@pytest.mark.parametrize("cfg,N,win,beta,ref", [(0, 10, (5, 11, 1, 1), 0.05, 0), (0, 10, (5, 11, 1, 1), 0.3, 4),
                                               (1, 15, (5, 11, 3, 6), 0.1, 0), (0, 20, (5, 11, 1, 1), 0.7, 19),
                                               (0, 6, (3, 5, 1, 1), 0.5, 2)])
def test_regularised_phase_link_parity(plk, ctx, cfg, N, win, beta, ref):
    z, m = case(cfg, N, 40, 70, win, seed=5 + N)
    C = oracle.covariance(z, win, m).astype(np.complex64)
    o = oracle.phase_link(C.astype(np.complex128), N, ref, beta=beta)
    g = ctx.phase_link(torch.from_numpy(C).cuda(), N, ref, plk.default_params(beta=beta))
    ph, tc, st = to_np(g["phase"]), to_np(g["tcoh"]), to_np(g["status"])
    live = o["status"] != 3
    assert np.array_equal(st == 3, ~live)
    clear = clear_of_degenerate(o, live)[0]
    assert clear.sum() >= 0.98 * live.sum()
    rep = phase_report(ph, o["phase"], clear)
    print(f"beta={beta}, N={N}: phase {rep}, EVD fallback {np.sum(o['status'] == 2)} of {live.sum()}")
    assert rep["max"] <= PHASE_TOL, rep
    assert np.nanmax(np.abs(tc[live] - o["tcoh"][live])) <= TCOH_TOL


@pytest.mark.parametrize("mu", [0.5, 1.2, 3.0])
def test_shift_above_or_below_lambda_min(plk, ctx, mu):
    # A caller's shift far below lambda_min converges slowly but to the same
    # eigenvector; one above it (lambda_min is near 1 without regularisation)
    # must not converge to the eigenvalue nearest the shift.
    N, win, ref = 10, (5, 11, 1, 1), 0
    z, m = case(0, N, 40, 70, win, seed=9)
    C = oracle.covariance(z, win, m).astype(np.complex64)
    o = oracle.phase_link(C.astype(np.complex128), N, ref)
    g = ctx.phase_link(torch.from_numpy(C).cuda(), N, ref, plk.default_params(mu=mu))
    ph, st = to_np(g["phase"]), to_np(g["status"])
    live = o["status"] != 3
    clear = clear_of_degenerate(o, live)[0] & (st != 4)
    assert clear.sum() >= 0.98 * live.sum()
    rep = phase_report(ph, o["phase"], clear)
    print(f"mu={mu}: phase {rep}, not converged {np.sum(st == 4)}")
    assert rep["max"] <= PHASE_TOL, rep


def good_weights(o, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1, 1, o["phase"].shape)
    bad = (np.abs(o["phase"]) > np.pi - 0.05).any(axis=0) | (o["status"] != 0) | \
          (o["gap"] < 1e-3 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
    w[:, bad] = 0.0
    return w.astype(np.float32), bad


@pytest.mark.parametrize("N,win,beta,ref", [(8, (5, 11, 1, 1), 0.2, 0), (12, (3, 5, 1, 1), 0.6, 5)])
def test_regularised_adjoint_matches_oracle_finite_differences(plk, ctx, N, win, beta, ref):
    H, W = 14, 26
    z, m = case(4, N, H, W, win, seed=70 + N)
    o = oracle.phase_link(oracle.covariance(z, win, m), N, ref, beta=beta)
    w, bad = good_weights(o, N)
    assert (~bad).sum() >= bad.size // 2
    prm = plk.default_params(beta=beta)
    g = to_np(ctx.phase_link_backward(torch.from_numpy(z).cuda(), win, torch.from_numpy(m.view(np.int64)).cuda(),
                                      ref, torch.from_numpy(w).cuda(), prm))

    def loss(zz):
        return float(np.sum(w * oracle.phase_link(oracle.covariance(zz, win, m), N, ref, beta=beta)["phase"]))

    rng = np.random.default_rng(N)
    h = 1e-6
    zd = z.astype(np.complex128)
    errs, refs = [], []
    for _ in range(24):
        i, y, x = rng.integers(N), rng.integers(H), rng.integers(W)
        for comp in (1.0, 1j):
            zp, zm = zd.copy(), zd.copy()
            zp[i, y, x] += h * comp
            zm[i, y, x] -= h * comp
            fd = (loss(zp) - loss(zm)) / (2 * h)
            ad = g[i, y, x].real if comp == 1.0 else g[i, y, x].imag
            errs.append(abs(ad - fd))
            refs.append(abs(fd))
    errs, refs = np.array(errs), np.array(refs)
    print(f"beta={beta}: adjoint vs oracle FD max abs err {errs.max():.3e}, max |grad| {refs.max():.3e}")
    assert np.all(errs <= 1e-3 * max(refs.max(), 1e-6) + 5e-3 * refs)


def test_regularised_uncertainty_and_weight_gradient(plk, ctx):
    N, win, ref, beta, H, W = 9, (5, 11, 5, 11), 3, 0.4, 5, 22
    z, m = case(4, N, H, W, win, seed=13)
    o = oracle.phase_link(oracle.covariance(z, win, m), N, ref, beta=beta)
    w, bad = good_weights(o, 2)
    assert not bad.any()
    prm = plk.default_params(beta=beta)
    zg, mg = torch.from_numpy(z).cuda(), torch.from_numpy(m.view(np.int64)).cuda()
    sd = to_np(ctx.phase_uncertainty(zg, win, mg, ref, 0.01, prm))
    dw = to_np(ctx.shp_weight_gradient(zg, win, mg, ref, torch.from_numpy(w).cuda(), prm))

    def phases(zz):
        return oracle.phase_link(oracle.covariance(zz, win, m), N, ref, beta=beta)["phase"]

    # uncertainty: the gradient norm of every phase by central differences over every sample
    h = 1e-6
    zd = z.astype(np.complex128)
    acc = np.zeros_like(o["phase"])
    for k in range(N):
        for y in range(H):
            for x in range(W):
                for comp in (1.0, 1j):
                    zp, zm = zd.copy(), zd.copy()
                    zp[k, y, x] += h * comp
                    zm[k, y, x] -= h * comp
                    d = (phases(zp) - phases(zm)) / (2 * h)
                    acc += d * d
    want = np.sqrt(0.5 * 0.01 * acc)
    np.testing.assert_allclose(sd, want, rtol=1e-2, atol=1e-4 * np.median(want))
    # weight gradient: one pixel's weights through the oracle's weighted coherence
    nb = win[0] * win[1]
    for ox in range(W // 11):
        s, inside = oracle.window_samples(zd, win, 0, ox)
        wts = oracle.mask_weights(m[0, ox], nb)
        for b in range(0, nb, 5):
            wp, wm = wts.copy(), wts.copy()
            wp[b] += h
            wm[b] -= h
            lp = oracle.phase_link(oracle.weighted_coherence(s, wp)[None], N, ref, beta=beta)["phase"][:, 0]
            lm = oracle.phase_link(oracle.weighted_coherence(s, wm)[None], N, ref, beta=beta)["phase"][:, 0]
            fd = float(np.dot(w[:, 0, ox], (lp - lm) / (2 * h)))
            assert abs(dw[0, ox, b] - fd) <= 1e-3 * max(abs(fd), 1e-2) + 2e-5, (ox, b, dw[0, ox, b], fd)
