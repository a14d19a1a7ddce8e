"""First-order phase uncertainty through the adjoint (plk_phase_uncertainty).

Under white circular Gaussian noise of variance sigma2 on every SLC sample
(E|n|^2 = sigma2, SHP masks frozen), the linearised variance of a linked
phase is (sigma2 / 2) times the squared norm of its gradient over the samples.

- Against the FP64 oracle: the gradient of every oracle phase by central
  finite differences over every sample of the image (real and imaginary
  parts), the variance formed from it; three date counts (the 8-, 16- and
  32-lane groups of the kernel), overlapping and tiling windows, a nonzero
  reference date.
- Against Monte Carlo of the oracle: noisy copies of one window with a small
  sigma, the sample standard deviation of the oracle's phase errors (this pins
  the sigma2 / 2 convention to what the noise actually does).
- Against the library's own adjoint (plk_phase_link_backward with the weight
  1 on one date): on tiling windows the gradients of different output pixels
  fall on disjoint samples, so the per-window squared norm is the variance.
- Exact properties: 0 at the reference date, NaN where the pixel has no data,
  proportional to sqrt(sigma2).
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


def stack(N, H, W, win, seed):
    z = synth.generate(synth.config_spec(4, N=N, H=H, W=W, seed=seed)).numpy()
    P, _ = oracle.amp_stats(z)
    m, _ = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    return z, m


def oracle_phases(z, win, m, N, ref):
    return oracle.phase_link(oracle.covariance(z, win, m), N, ref)


def oracle_sd_by_fd(z, win, m, N, ref, sigma2, h=1e-6):
    """sqrt((sigma2 / 2) sum over samples of |d phase / d Re z|^2 + |d phase / d Im z|^2)."""
    zd = z.astype(np.complex128)
    acc = None
    for k in range(N):
        for y in range(z.shape[1]):
            for x in range(z.shape[2]):
                for comp in (1.0, 1j):
                    zp, zm = zd.copy(), zd.copy()
                    zp[k, y, x] += h * comp
                    zm[k, y, x] -= h * comp
                    d = (oracle_phases(zp, win, m, N, ref)["phase"] -
                         oracle_phases(zm, win, m, N, ref)["phase"]) / (2 * h)
                    acc = d * d if acc is None else acc + d * d
    return np.sqrt(0.5 * sigma2 * acc)


def well_posed(o):
    """Pixels whose phases are away from the wrap and whose eigenvector is unique."""
    return ~((np.abs(o["phase"]) > np.pi - 0.05).any(axis=0) | (o["status"] == 3) |
             (o["gap"] < 1e-3 * np.abs(np.nan_to_num(o["lam"], nan=1.0))))


def gpu_sd(ctx, z, m, win, ref, sigma2):
    return to_np(ctx.phase_uncertainty(torch.from_numpy(z).cuda(), win,
                                       torch.from_numpy(m.view(np.int64)).cuda(), ref, sigma2))


@pytest.mark.parametrize("N,H,W,win,ref", [(6, 8, 16, (3, 5, 1, 1), 5),      # 8-lane groups, overlapping
                                           (12, 5, 22, (5, 11, 5, 11), 4),   # 16-lane groups, tiling
                                           (24, 5, 11, (5, 11, 5, 11), 0)])  # 32-lane groups
def test_uncertainty_matches_oracle_gradient_norm(ctx, plk, N, H, W, win, ref):
    z, m = stack(N, H, W, win, seed=11 + N)
    sigma2 = 0.01
    o = oracle_phases(z, win, m, N, ref)
    want = oracle_sd_by_fd(z, win, m, N, ref, sigma2)
    got = gpu_sd(ctx, z, m, win, ref, sigma2)
    ok = well_posed(o)
    assert ok.sum() >= max(1, ok.size // 2)
    assert np.all(got[ref] == 0.0)
    err = np.abs(got - want)[:, ok]
    scale = np.median(want[:, ok])
    print(f"N={N}: max rel err {np.max(err / np.maximum(want[:, ok], 1e-12)):.3e}, median sd {scale:.3e}")
    assert np.all(err <= 1e-2 * want[:, ok] + 1e-4 * scale)


def test_uncertainty_matches_oracle_monte_carlo(ctx, plk):
    # One 5 x 11 window, K noisy copies side by side as K tiling output pixels
    # of one oracle call, each with the same frozen mask.
    N, win, ref, K = 8, (5, 11, 5, 11), 2, 4000
    z, m = stack(N, 5, 11, win, seed=3)
    o = oracle_phases(z, win, m, N, ref)
    assert well_posed(o).all()
    sigma = 1e-3 * np.sqrt(np.mean(np.abs(z) ** 2))
    rng = np.random.default_rng(4)
    zk = np.tile(z.astype(np.complex128), (1, 1, K))
    zk += (sigma / np.sqrt(2)) * (rng.standard_normal(zk.shape) + 1j * rng.standard_normal(zk.shape))
    mk = np.tile(m, (1, K, 1))
    ph = oracle_phases(zk, win, mk, N, ref)["phase"].reshape(N, K)
    dev = np.angle(np.exp(1j * (ph - o["phase"].reshape(N, 1))))
    mc = dev.std(axis=1)
    got = gpu_sd(ctx, z, m, win, ref, sigma ** 2)[:, 0, 0]
    print("Monte Carlo sd", mc, "predicted", got)
    assert got[ref] == 0.0 and mc[ref] == 0.0
    others = [i for i in range(N) if i != ref]
    # sample sd of K draws: relative standard error 1/sqrt(2K) ~ 1.1 %
    assert np.all(np.abs(got[others] - mc[others]) <= 0.06 * mc[others])


@pytest.mark.parametrize("N", [10, 20, 32])
def test_uncertainty_equals_backward_gradient_norm(ctx, plk, N):
    win, ref, H, W = (5, 11, 5, 11), N // 3, 40, 88
    z, m = stack(N, H, W, win, seed=60 + N)
    sigma2 = 0.5
    zg = torch.from_numpy(z).cuda()
    mg = torch.from_numpy(m.view(np.int64)).cuda()
    got = gpu_sd(ctx, z, m, win, ref, sigma2)
    Ho, Wo = H // 5, W // 11
    for i in range(N):
        if i == ref:
            assert np.all(got[i] == 0.0)
            continue
        w = torch.zeros((N, Ho, Wo), dtype=torch.float32, device="cuda")
        w[i] = 1.0
        g = to_np(ctx.phase_link_backward(zg, win, mg, ref, w)).astype(np.complex128)
        norm2 = (np.abs(g) ** 2).sum(axis=0).reshape(Ho, 5, Wo, 11).sum(axis=(1, 3))
        want = np.sqrt(0.5 * sigma2 * norm2)
        np.testing.assert_allclose(got[i], want, rtol=2e-3, atol=1e-6 * want.max())


def test_no_data_pixel_scaling_and_reference(ctx, plk):
    N, win, ref, H, W = 9, (5, 11, 5, 11), 3, 10, 33
    z, _ = stack(N, H, W, win, seed=8)
    z[:, 5:10, 11:22] = 0                       # output pixel (1, 1): no sample passes the SHP test
    P, _ = oracle.amp_stats(z)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    assert cnt[1, 1] == 0
    o = oracle_phases(z, win, m, N, ref)
    assert o["status"][1, 1] == 3
    a = gpu_sd(ctx, z, m, win, ref, 0.3)
    b = gpu_sd(ctx, z, m, win, ref, 1.2)
    assert np.all(np.isnan(a[:, 1, 1])) and np.all(np.isnan(b[:, 1, 1]))
    live = np.ones((H // 5, W // 11), bool)
    live[1, 1] = False
    assert np.all(a[ref][live] == 0.0)
    np.testing.assert_allclose(b[:, live], 2.0 * a[:, live], rtol=1e-6)
    assert np.all(a[:, live] >= 0.0) and np.all(np.isfinite(a[:, live]))


def test_uncertainty_rejects_bad_arguments(ctx, plk):
    N, win = 6, (3, 5, 1, 1)
    z, m = stack(N, 8, 16, win, seed=1)
    zg = torch.from_numpy(z).cuda()
    mg = torch.from_numpy(m.view(np.int64)).cuda()
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(plk.PlkError):
            ctx.phase_uncertainty(zg, win, mg, 0, bad)
    with pytest.raises(plk.PlkError):
        ctx.phase_uncertainty(zg, win, mg, N, 0.1)
