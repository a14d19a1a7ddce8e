"""L1 network inversion by ADMM on the GPU (plk_invert_l1) against the
oracle on the same seeded unwrapped phases.

Bars: x and the residual b - A x within 2e-4 rad per unit of the phases' scale
after the same number of iterations (single against double precision; the
ADMM map is non-expansive, so rounding does not grow with the iterations);
sparse 2 pi unwrapping errors rejected as by the oracle; the network checks."""
import numpy as np
import pytest
import torch

import oracle
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


def unwrapped(pairs, n_dates, npx, seed, err_frac=0.03, noise=0.3):
    rng = np.random.default_rng(seed)
    A = oracle.incidence(pairs, n_dates)
    xt = np.cumsum(rng.normal(0, 1.5, (n_dates - 1, npx)), axis=0)
    k = np.where(rng.random((len(pairs), npx)) < err_frac, rng.choice([-1, 1], (len(pairs), npx)), 0)
    b = A @ xt + 2 * np.pi * k + rng.normal(0, noise, (len(pairs), npx))
    return b.astype(np.float32), xt, k


@pytest.mark.parametrize("n_dates,which,npx,rho,iters", [
    (15, "n3", 3000, 1.0, 50), (15, "n3", 1000, 0.5, 200), (8, "n3", 777, 2.0, 30), (17, "n3", 513, 1.0, 40),
    (12, "n2", 900, 1.0, 25), (10, "sub", 640, 1.0, 60), (2, "n3", 300, 1.0, 5), (15, "n3", 200, 1.0, 1)])
def test_invert_l1_parity(ctx, plk, n_dates, which, npx, rho, iters):
    pairs = oracle.nearest3_pairs(n_dates)
    if which == "n2":
        pairs = [p for p in pairs if p[1] - p[0] <= 2]
    elif which == "sub":  # a nearest-3 subset in scrambled order: every (a, a+1) and some longer pairs
        rng = np.random.default_rng(1)
        pairs = [p for p in pairs if p[1] - p[0] == 1 or rng.random() < 0.5]
        pairs = [pairs[i] for i in rng.permutation(len(pairs))]
    b, xt, k = unwrapped(pairs, n_dates, npx, seed=n_dates + iters)
    o = oracle.l1_invert(b.astype(np.float64), pairs, n_dates, rho, iters)
    x, r = ctx.invert_l1(torch.from_numpy(b).cuda(), n_dates, pairs, rho=rho, iters=iters, residual=True)
    x, r = to_np(x), to_np(r)
    scale = max(1.0, float(np.abs(b).max()))
    ex = np.abs(x - o["x"]).max() / scale
    er = np.abs(r - o["residual"]).max() / scale
    print(f"N={n_dates} {which} npx={npx} rho={rho} iters={iters}: max |x - oracle| / scale {ex:.2e}, "
          f"residual {er:.2e}")
    assert ex <= 2e-4 and er <= 2e-4


def test_invert_l1_rejects_sparse_unwrapping_errors(ctx, plk):
    pairs = oracle.nearest3_pairs(15)
    b, xt, k = unwrapped(pairs, 15, 4096, seed=7, err_frac=0.02, noise=0.0)
    x, r = ctx.invert_l1(torch.from_numpy(b).cuda(), 15, pairs, rho=1.0, iters=200, residual=True)
    x, r = to_np(x), to_np(r)
    one = (np.abs(k).sum(axis=0) <= 1)              # pixels with at most one wrong interferogram
    assert one.mean() > 0.8
    assert np.abs(x - xt)[:, one].max() < 1e-3
    assert np.abs(r - 2 * np.pi * k)[:, one].max() < 1e-3


def test_invert_l1_network_checks(ctx, plk):
    b = torch.zeros((3, 10), device="cuda")
    with pytest.raises(plk.PlkError):
        ctx.invert_l1(b, 5, [(0, 1), (1, 2), (0, 4)])          # b - a = 4: outside nearest-3
    with pytest.raises(plk.PlkError):
        ctx.invert_l1(b, 4, [(0, 1), (0, 1), (1, 3)])          # repeated pair
    with pytest.raises(plk.PlkError):
        ctx.invert_l1(b, 5, [(0, 1), (1, 2), (2, 3)])          # date 4 undetermined
    with pytest.raises(plk.PlkError):
        ctx.invert_l1(b, 4, [(0, 1), (1, 2), (2, 3)], rho=0.0)  # rho must be positive
    with pytest.raises(plk.PlkError):
        ctx.invert_l1(torch.zeros((17, 4), device="cuda"), 18, [(a, a + 1) for a in range(17)])  # > 17 dates
    # two dates, one interferogram: x = b exactly
    bb = torch.linspace(-5, 5, 50, device="cuda").view(1, 50)
    assert torch.allclose(ctx.invert_l1(bb, 2, [(0, 1)], iters=3), bb)
