"""Persistent scatterers on the GPU (plk_ps_regrid; ps_da_max in
plk_ministack_step) against the oracle on the same seeded inputs.

Bars: PS flags and cell statuses bit-exact (D_A decided in single precision,
correctly rounded, on both sides); cells without PS untouched bit for bit;
PS phases within 1e-5 rad (wrapped); compressed SLCs within single-precision
accumulation error; a planted PS keeps the scheme's datum along the chain."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import PHASE_TOL, TCOH_TOL, count_np, phase_report, to_np, wrapped_diff, write_state_file

pytestmark = pytest.mark.gpu

PS_PHASE_TOL = 1e-5


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


def ps_stack(N, H, W, seed, frac=0.05):
    # the burst workload's PS population (amplitude 3 (1 + eps), eps ~ CN(0, 0.1^2):
    # D_A near 0.07) in its DS background, plus exact-dispersion planted pixels
    spec = synth.config_spec(1, N=N, H=H, W=W, seed=seed, ps_fraction=frac)
    z = synth.generate(spec).numpy()
    rng = np.random.default_rng(seed)
    ys, xs = rng.integers(0, H, 12), rng.integers(0, W, 12)
    # amplitudes 1, 1.5 alternating with phases on multiples of pi/2, so |z| is
    # exact: D_A = 0.2 exactly over an even number of dates (on the threshold)
    amps = np.where(np.arange(N) % 2 == 0, 1.0, 1.5)
    quarter = np.array([1, 1j, -1, -1j], np.complex64)
    for y, x in zip(ys, xs):
        z[:, y, x] = amps.astype(np.float32) * quarter[rng.integers(0, 4, N)]
    z[:, ys[0], xs[0]] = 0                                  # no amplitude
    z[N // 2, ys[1], xs[1]] = 0                             # one zero sample
    return z


@pytest.mark.parametrize("N,H,W,win,first_real,da_max", [
    (15, 61, 203, (5, 11, 3, 6), 0, 0.2),      # the burst strides; ragged rows and columns
    (17, 40, 97, (5, 11, 3, 6), 3, 0.2),       # a mini-stack: 3 compressed SLCs, reference entry 2
    (10, 37, 64, (5, 11, 1, 1), 0, 0.25),      # full-resolution output
    (8, 33, 71, (3, 5, 2, 5), 2, 0.15),        # odd strides, a stricter threshold
])
def test_ps_regrid_parity(ctx, plk, N, H, W, win, first_real, da_max):
    z = ps_stack(N, H, W, seed=N + H)
    ref = max(first_real - 1, 0)
    Ho, Wo = H // win[2], W // win[3]
    sp, sa = oracle.amp_stats(z[first_real:])
    rng = np.random.default_rng(1)
    ds_phase = rng.uniform(-np.pi, np.pi, (N - first_real, Ho, Wo)).astype(np.float32)
    ds_status = rng.integers(0, 5, (Ho, Wo)).astype(np.uint8)
    ph_o, st_o = oracle.ps_regrid(z, first_real, win, sp, sa, N - first_real, ref, da_max, ds_phase, ds_status)
    ph_g = torch.from_numpy(ds_phase.copy()).cuda()
    st_g = torch.from_numpy(ds_status.copy()).cuda()
    ctx.ps_regrid(torch.from_numpy(z).cuda(), first_real, win, torch.from_numpy(sp).cuda(),
                  torch.from_numpy(sa).cuda(), N - first_real, ref, da_max, ph_g, st_g)
    st_g, ph_g = to_np(st_g), to_np(ph_g)
    assert np.array_equal(st_g, st_o)
    ps = st_o == plk.PX_PS
    assert 0 < ps.sum() < ps.size
    assert np.array_equal(ph_g[:, ~ps], ds_phase[:, ~ps])
    err = wrapped_diff(ph_g[:, ps], ph_o[:, ps])
    print(f"PS cells {ps.sum()} of {ps.size}; max PS phase error {err.max():.2e} rad")
    assert err.max() <= PS_PHASE_TOL
    if ref >= first_real:  # the reference is a real date: its PS phase is exactly zero
        assert np.all(ph_g[ref - first_real][ps] == 0.0)


def test_ps_regrid_reference_date_is_exactly_zero(ctx, plk):
    z = ps_stack(12, 30, 60, seed=4)
    sp, sa = oracle.amp_stats(z)
    win = (5, 11, 3, 6)
    ph = torch.zeros((12, 10, 10), device="cuda")
    st = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    ctx.ps_regrid(torch.from_numpy(z).cuda(), 0, win, torch.from_numpy(sp).cuda(), torch.from_numpy(sa).cuda(),
                  12, 4, 0.2, ph, st)
    ps = to_np(st) == plk.PX_PS
    assert ps.any() and np.all(to_np(ph)[4][ps] == 0.0)


def test_ps_regrid_threshold_zero_and_rejections(ctx, plk):
    z = ps_stack(6, 12, 24, seed=5)
    zg = torch.from_numpy(z).cuda()
    sp, sa = (torch.from_numpy(a).cuda() for a in oracle.amp_stats(z))
    ph = torch.full((6, 4, 4), 9.0, device="cuda")
    st = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    ctx.ps_regrid(zg, 0, (3, 5, 3, 6), sp, sa, 6, 0, 0.0, ph, st)   # D_A = 0 exactly: none here
    assert torch.all(st == 0) and torch.all(ph == 9.0)
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(plk.PlkError):
            ctx.ps_regrid(zg, 0, (3, 5, 3, 6), sp, sa, 6, 0, bad, ph, st)
    with pytest.raises(plk.PlkError):
        ctx.ps_regrid(zg, 0, (3, 5, 3, 6), sp, sa, 6, 6, 0.2, ph, st)      # ref out of range
    st_ = plk.State(ctx, 12, 24, (3, 5, 3, 6), K_max=1, M_max=6)
    with pytest.raises(plk.PlkError):
        st_.step(zg, plk.default_params(ps_da_max=-1.0))
    st_.close()


def test_ps_regrid_fallback_when_lowest_fails_its_check(ctx, plk):
    # Per block, the pixel of lowest D_A has a zero sample (standalone call:
    # on a real date, where the merged sums still give it the lowest D_A) or
    # a zero reference sample; the next lowest must be taken, as the oracle does.
    N, H, W, win = 31, 6, 24, (3, 5, 3, 6)
    rng = np.random.default_rng(7)
    z = (rng.standard_normal((N, H, W)) + 1j * rng.standard_normal((N, H, W))).astype(np.complex64)
    t = np.arange(N)
    for cj in range(4):
        ya, xa, yb, xb = 0, 6 * cj + 1, 2, 6 * cj + 4
        z[:, ya, xa] = (2.0 * np.exp(0.3j * t)).astype(np.complex64)
        z[5, ya, xa] = 0                        # one zero sample: D_A = 1/sqrt(30) = 0.1826, the lowest
        z[:, yb, xb] = (np.where(t % 2 == 0, 1.0, 1.45) * np.exp(-0.2j * t)).astype(np.complex64)  # 0.1837
    z[0, 3, 2] = 0                              # cell (1, 0): a zero reference sample at its best pixel
    z[:, 3, 2] = (3.0 * np.exp(0.1j * t)).astype(np.complex64) * (t > 0)
    z[:, 5, 3] = (np.where(t % 2 == 0, 1.0, 1.45) * np.exp(0.5j * t)).astype(np.complex64)
    sp, sa = oracle.amp_stats(z)
    Ho, Wo = 2, 4
    ph0 = np.zeros((N, Ho, Wo), np.float32)
    st0 = np.zeros((Ho, Wo), np.uint8)
    ph_o, st_o = oracle.ps_regrid(z, 0, win, sp, sa, N, 0, 0.2, ph0, st0)
    want = np.zeros((Ho, Wo), bool)
    want[0, :] = want[1, 0] = True
    assert np.array_equal(st_o == plk.PX_PS, want)
    ph_g = torch.from_numpy(ph0.copy()).cuda()
    st_g = torch.from_numpy(st0.copy()).cuda()
    ctx.ps_regrid(torch.from_numpy(z).cuda(), 0, win, torch.from_numpy(sp).cuda(), torch.from_numpy(sa).cuda(),
                  N, 0, 0.2, ph_g, st_g)
    assert np.array_equal(to_np(st_g), st_o)
    assert wrapped_diff(to_np(ph_g), ph_o).max() <= PS_PHASE_TOL
    assert wrapped_diff(ph_o[:, 0, :], (-0.2 * t)[:, None]).max() < 1e-5
    assert wrapped_diff(ph_o[:, 1, 0], 0.5 * t).max() < 1e-5


def test_ministack_ps_fallback_on_zero_compressed_sample(plk, ctx, tmp_path):
    # Inside a step (dispersions from the S1 plane): the newest compressed SLC
    # is zero at a block's lowest-D_A pixel, so the next lowest is taken.
    z = ps_stack(20, 24, 60, seed=21)
    win = (5, 11, 3, 6)
    orc = oracle.OracleChain(24, 60, win, K_max=2, alpha=1e-3, kappa_dtype=np.complex64, ps_da_max=0.2)
    orc.step(z[:10])
    sa = orc.sum_amp.copy()
    sp = orc.sum_pow.copy()
    da = oracle.amp_dispersion(sp, sa, 10)
    blk = da[:3, :6].astype(np.float64)
    y, x = np.unravel_index(int(np.nanargmin(blk)), blk.shape)
    assert blk[y, x] <= 0.2
    orc.ring[-1][y, x] = 0                      # the lowest-D_A pixel of cell (0, 0) loses its reference
    path = str(tmp_path / "s.plk")
    write_state_file(path, orc)
    st = plk.State.load(ctx, path, M_max=10)
    g = st.step(torch.from_numpy(z[10:]).cuda().contiguous(), plk.default_params(ps_da_max=0.2))
    o = orc.step(z[10:])
    assert np.array_equal(to_np(g["status"]) == plk.PX_PS, o["status"] == plk.PX_PS)
    ps = o["status"] == plk.PX_PS
    assert wrapped_diff(to_np(g["phase"])[:, ps], o["phase"][1:][:, ps]).max() <= PS_PHASE_TOL
    st.close()


def chain_case(scheme_seed):
    z = ps_stack(30, 48, 150, seed=scheme_seed)
    return torch.from_numpy(z), (5, 11, 3, 6), 10, 2, 30


@pytest.mark.parametrize("scheme", ["first", "last"])
def test_ministack_step_ps_parity(plk, ctx, scheme, tmp_path):
    """Each step from identical inputs (the oracle's state loaded through the
    checkpoint format): statuses with the PS code bit-exact, DS phases within
    the phase tolerance, PS phases within 1e-5, the new compressed SLC with its
    PS pixels compressed on their own phases."""
    z, window, M, K_max, nd = chain_case(11 if scheme == "first" else 12)
    H, W = z.shape[1:]
    orc = oracle.OracleChain(H, W, window, K_max=K_max, alpha=1e-3, kappa_dtype=np.complex64, scheme=scheme,
                             ps_da_max=0.2)
    prm = plk.default_params(ps_da_max=0.2, ref_scheme=plk.REF_LAST_REAL if scheme == "last" else plk.REF_FIRST)
    zg = z.cuda()
    for k, sl in enumerate(synth.ministack_slices(nd, M)):
        path = str(tmp_path / f"s{k}.plk")
        write_state_file(path, orc)
        st = plk.State.load(ctx, path, M_max=M)
        g = st.step(zg[sl].contiguous(), prm)
        o = orc.step(z[sl].numpy())
        assert np.array_equal(count_np(g["count"]), o["count"]), k
        st_g = to_np(g["status"])
        ps = o["status"] == plk.PX_PS
        assert np.array_equal(st_g == plk.PX_PS, ps), k
        assert 0.3 * ps.size < ps.sum() < ps.size
        K = o["K_used"]
        pg, po = to_np(g["phase"]), o["phase"][K:]
        assert wrapped_diff(pg[:, ps], po[:, ps]).max() <= PS_PHASE_TOL, k
        live = (o["status"] != 3) & ~ps
        clear = live & (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
        rep = phase_report(pg, po, clear)
        assert rep["max"] <= PHASE_TOL, (k, rep)
        tg = to_np(g["tcoh"])
        assert np.array_equal(np.isnan(tg), np.isnan(o["tcoh"]))
        assert np.nanmax(np.abs(tg - o["tcoh"])) <= TCOH_TOL
        kg = to_np(st.kappa(st.info()["K_used"] - 1))
        scale = np.abs(z[sl].numpy()).sum(0)
        assert np.max(np.abs(kg - orc.ring[-1]) / (scale + 1e-6)) < 1e-4, k
        st.close()


@pytest.mark.parametrize("scheme", ["first", "last"])
def test_chain_planted_ps_keeps_datum(plk, ctx, scheme):
    # A PS with its own phase history in a noise-free DS background (whose
    # amplitudes alternate 0.2 a / 1.8 a: D_A near 0.8, never a PS).
    n_dates, M, H, W, win = 20, 5, 24, 48, (3, 5, 3, 6)
    t = np.arange(n_dates)
    phi_ds, phi_ps = 0.2 * t, 0.9 * t + 0.5 * np.sin(t)
    rng = np.random.default_rng(10)
    a = rng.uniform(0.5, 2.0, (H, W))
    lo = rng.integers(0, 2, (H, W))
    amp = np.where((t[:, None, None] + lo[None]) % 2 == 0, 0.2, 1.8) * a[None]
    z = amp * np.exp(1j * (phi_ds[:, None, None] + rng.uniform(-np.pi, np.pi, (H, W))[None]))
    z[:, 7, 20] = 3.0 * np.exp(1j * (phi_ps + 1.3))                 # cell (2, 3)
    zg = torch.from_numpy(z.astype(np.complex64)).cuda()
    st = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    prm = plk.default_params(ps_da_max=0.2, ref_scheme=plk.REF_LAST_REAL if scheme == "last" else plk.REF_FIRST)
    for s, sl in enumerate(synth.ministack_slices(n_dates, M)):
        g = st.step(zg[sl].contiguous(), prm)
        sg = to_np(g["status"])
        assert sg[2, 3] == plk.PX_PS and np.sum(sg == plk.PX_PS) == 1
        ref_date = 0 if (s == 0 or scheme == "first") else sl.start - 1
        want_ps = phi_ps[sl] - phi_ps[ref_date]
        assert wrapped_diff(to_np(g["phase"])[:, 2, 3], want_ps).max() < 1e-4, s
        want_ds = (phi_ds[sl] - phi_ds[ref_date])[:, None, None]
        ds = sg != plk.PX_PS
        assert wrapped_diff(to_np(g["phase"]), np.broadcast_to(want_ds, g["phase"].shape))[:, ds].max() < 1e-4, s
    st.close()


def test_ps_off_changes_nothing(plk, ctx):
    # ps_da_max = 0 (the default) leaves the step bit-identical to a step
    # without the field.
    z = torch.from_numpy(ps_stack(15, 48, 120, seed=3)).cuda()
    outs = []
    for prm in (None, plk.default_params(ps_da_max=0.0)):
        st = plk.State(ctx, 48, 120, (5, 11, 3, 6), K_max=2, M_max=15)
        outs.append((st.step(z, prm), to_np(st.kappa(0))))
        st.close()
    (a, ka), (b, kb) = outs
    for key in ("phase", "tcoh", "status"):
        assert torch.equal(torch.nan_to_num(a[key].float(), nan=-9.0), torch.nan_to_num(b[key].float(), nan=-9.0))
    assert np.array_equal(ka, kb)
