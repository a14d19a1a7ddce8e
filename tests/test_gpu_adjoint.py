"""Adjoint of coherence -> EMI -> referenced phase (plk_phase_link_backward,
PhaseLinkFn), SHP masks frozen.  L = sum w * phase.

- Exact identities of the method: a per-date phase screen z_i -> z_i e^{j b_i}
  shifts phase_i by b_i - b_ref, so the derivative of L along j z_i is the sum
  of date i's weights (minus all weights for the reference date); scaling a
  date leaves the coherence unchanged, so the derivative along z_i is 0.
- Central finite differences of the FP64 oracle (h = 1e-6) on sampled
  elements: the oracle gradient.
- Central finite differences (h = 1e-3) of the library's own single-precision
  forward pass on sampled elements.
- The autograd Function gives the same gradient as the entry point."""
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
    spec = synth.config_spec(4, N=N, H=H, W=W, seed=seed)
    z = synth.generate(spec).numpy()
    P, _ = oracle.amp_stats(z)
    m, _ = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    C = oracle.covariance(z, win, m)
    o = oracle.phase_link(C, N, ref)
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1, 1, o["phase"].shape)
    # no weight where the phase is near the wrap or the eigenvector is not unique
    bad = (np.abs(o["phase"]) > np.pi - 0.05).any(axis=0) | (o["status"] == 3) | \
          (o["gap"] < 1e-3 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
    w[:, bad] = 0.0
    return z, m, w.astype(np.float32), o


def oracle_loss(z, m, win, N, ref, w):
    C = oracle.covariance(z, win, m)
    return float(np.sum(w * oracle.phase_link(C, N, ref)["phase"]))


def gpu_grad(ctx, z, m, win, ref, w):
    g = ctx.phase_link_backward(torch.from_numpy(z).cuda(), win, torch.from_numpy(m.view(np.int64)).cuda(), ref,
                                torch.from_numpy(w).cuda())
    return to_np(g)


@pytest.mark.parametrize("N,win,ref", [(10, (5, 11, 1, 1), 0), (20, (5, 11, 1, 1), 7), (15, (5, 11, 3, 6), 0),
                                       (6, (3, 5, 1, 1), 5)])
def test_adjoint_equivariance_identities(ctx, plk, N, win, ref):
    z, m, w, o = case(N, 30, 60, win, seed=3 + N, ref=ref)
    g = gpu_grad(ctx, z, m, win, ref, w).astype(np.complex128)
    zc = z.astype(np.complex128)
    live = o["status"] != 3
    wl = np.where(live[None], w, 0.0)
    W_tot = wl.sum(axis=(1, 2))
    scale = np.sqrt(np.mean(np.abs(g) ** 2)) * np.sqrt(np.mean(np.abs(zc) ** 2)) * zc[0].size
    for i in range(N):
        d_phase = float(np.sum(np.real(np.conj(g[i]) * (1j * zc[i]))))
        want = W_tot[i] if i != ref else -(W_tot.sum() - W_tot[ref])
        assert abs(d_phase - want) <= 2e-3 * max(1.0, abs(want)) + 1e-4 * scale, (i, d_phase, want)
        d_scale = float(np.sum(np.real(np.conj(g[i]) * zc[i])))
        assert abs(d_scale) <= 1e-4 * scale, (i, d_scale)


@pytest.mark.parametrize("N,win,ref", [(8, (5, 11, 1, 1), 0), (12, (3, 5, 1, 1), 4)])
def test_adjoint_matches_oracle_finite_differences(ctx, plk, N, win, ref):
    H, W = 14, 26
    z, m, w, o = case(N, H, W, win, seed=40 + N, ref=ref)
    g = gpu_grad(ctx, z, m, win, ref, w)
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
            fd = (oracle_loss(zp, m, win, N, ref, w) - oracle_loss(zm, m, win, N, ref, w)) / (2 * h)
            ad = g[i, y, x].real if comp == 1.0 else g[i, y, x].imag
            errs.append(abs(ad - fd))
            refs.append(abs(fd))
    errs, refs = np.array(errs), np.array(refs)
    tol = 1e-3 * max(refs.max(), 1e-6) + 5e-3 * refs
    print(f"adjoint vs oracle FD: max abs err {errs.max():.3e}, max |grad| {refs.max():.3e}")
    assert np.all(errs <= tol), (errs - tol).max()


def test_adjoint_matches_library_finite_differences_and_autograd(ctx, plk):
    N, win, ref, H, W = 20, (5, 11, 1, 1), 0, 20, 32
    z, m, w, o = case(N, H, W, win, seed=77, ref=ref)
    zg = torch.from_numpy(z).cuda()
    mg = torch.from_numpy(m.view(np.int64)).cuda()
    wg = torch.from_numpy(w).cuda()
    # autograd through PhaseLinkFn
    zr = zg.clone().requires_grad_(True)
    ph = plk.PhaseLinkFn.apply(zr, mg, win, ref, ctx)
    (ph * wg).sum().backward()
    g_auto = to_np(zr.grad)
    g = gpu_grad(ctx, z, m, win, ref, w)
    # same computation; the scatter's shared-memory sums may add in another order
    assert np.allclose(g_auto, g, rtol=1e-5, atol=1e-6 * np.abs(g).max())

    def loss(zz):
        with torch.no_grad():
            return float((plk.PhaseLinkFn.apply(zz, mg, win, ref, ctx).double() * wg.double()).sum())

    rng = np.random.default_rng(1)
    h = 1e-3
    errs, refs = [], []
    for _ in range(16):
        i, y, x = rng.integers(N), rng.integers(H), rng.integers(W)
        for comp in (1.0, 1j):
            zp, zm = zg.clone(), zg.clone()
            zp[i, y, x] += h * comp
            zm[i, y, x] -= h * comp
            fd = (loss(zp) - loss(zm)) / (2 * h)
            ad = g[i, y, x].real if comp == 1.0 else g[i, y, x].imag
            errs.append(abs(ad - fd))
            refs.append(abs(fd))
    errs, refs = np.array(errs), np.array(refs)
    print(f"adjoint vs library FD (h=1e-3): max abs err {errs.max():.3e}, max |grad| {refs.max():.3e}")
    assert np.all(errs <= 2e-2 * max(refs.max(), 1e-3) + 2e-2 * refs)


def test_backward_rejects_small_workspace(ctx, plk):
    import ctypes
    L = plk.lib()
    z = torch.zeros((4, 16, 16), dtype=torch.complex64, device="cuda")
    out = torch.zeros_like(z)
    m = torch.zeros((16, 16, 1), dtype=torch.int64, device="cuda")
    dp = torch.zeros((4, 16, 16), device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    rc = L.plk_phase_link_backward(ctx.h, ctypes.c_void_p(z.data_ptr()), 4, 16, 16, plk.window((3, 3, 1, 1)),
                                   ctypes.c_void_p(m.data_ptr()), 0, None, ctypes.c_void_p(dp.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), 256, ctypes.c_void_p(out.data_ptr()))
    assert rc == 1
