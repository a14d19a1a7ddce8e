"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: SHP masks, counts and power sums bit-exact; linked phase within 1e-4 rad
(wrapped); temporal coherence within 1e-5; coherence and compressed SLCs within
single-precision accumulation error.  Sizes are small enough for the oracle to
finish in seconds but span several CTA tiles and ragged tails.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import (PHASE_TOL, TCOH_TOL, clear_of_degenerate, count_np, mask_np, phase_report, to_np,
                         wrapped_diff, write_state_file)

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


def stack(cfg, **over):
    spec = synth.config_spec(cfg, **over)
    return synth.generate(spec), spec


# ------------------------------------------------------------------ S1, S2

@pytest.mark.parametrize("shape", [(10, 64, 96), (15, 37, 53), (3, 1, 1)])
def test_amp_stats_bit_exact(ctx, shape):
    n, H, W = shape
    z, _ = stack(1, N=n, H=H, W=W, seed=7)
    P, A = oracle.amp_stats(z.numpy())
    zg = z.cuda()
    Pg, Ag = ctx.amp_stats(zg, sum_amp=torch.empty((H, W), device="cuda"))
    assert np.array_equal(to_np(Pg), P)
    assert np.array_equal(to_np(Ag), A)
    z2, _ = stack(0, N=4, H=H, W=W, seed=8)
    oracle.amp_stats(z2.numpy(), P, A, accumulate=True)
    ctx.amp_stats(z2.cuda(), Pg, Ag, accumulate=True)
    assert np.array_equal(to_np(Pg), P)
    assert np.array_equal(to_np(Ag), A)


@pytest.mark.parametrize("win", [(5, 11, 1, 1), (5, 11, 3, 6), (19, 37, 3, 6), (3, 3, 2, 2), (1, 1, 1, 1)])
def test_shp_select_bit_exact(ctx, win):
    z, spec = stack(1, N=15, H=61, W=134, seed=3)  # 5% persistent scatterers
    P, _ = oracle.amp_stats(z.numpy())
    P[7, 9:20] = 0.0  # a no-data streak
    c = oracle.glrt_threshold(1e-3, 15)
    m_o, n_o = oracle.shp_select(P, win, np.float32(c))
    m_g, n_g = ctx.shp_select(torch.from_numpy(P).cuda(), 15, win, 1e-3)
    assert np.array_equal(mask_np(m_g), m_o)
    assert np.array_equal(count_np(n_g), n_o)


# -------------------------------------------------------------------- S3

@pytest.mark.parametrize("cfg,N,win", [(0, 10, (5, 11, 1, 1)), (1, 15, (5, 11, 3, 6)), (0, 2, (3, 5, 1, 1)),
                                       (0, 21, (5, 11, 3, 6)), (0, 32, (5, 11, 3, 6)), (0, 18, (19, 37, 3, 6))])
def test_covariance_parity(ctx, cfg, N, win):
    z, _ = stack(cfg, N=N, H=50, W=97, seed=11)
    zn = z.numpy()
    P, _ = oracle.amp_stats(zn)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    C_o = oracle.covariance(zn, win, m)
    C_g = to_np(ctx.estimate_covariance(z.cuda(), win, torch.from_numpy(m.view(np.int64)).cuda()))
    ok = cnt > 0
    assert np.all(np.isnan(C_g[~ok].real))
    err = np.abs(C_g[ok] - C_o[ok])
    assert err.max() < 2e-5, err.max()


# ------------------------------------------------------------------ S4-S6

def oracle_C(cfg, N, H, W, win, seed, **over):
    z, _ = stack(cfg, N=N, H=H, W=W, seed=seed, **over)
    zn = z.numpy()
    P, _ = oracle.amp_stats(zn)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    C = oracle.covariance(zn, win, m)
    # Both sides link the same single-precision coherence.
    return C.astype(np.complex64)


@pytest.mark.parametrize("cfg,N,ref", [(0, 10, 0), (1, 15, 0), (0, 2, 1), (0, 5, 2), (0, 16, 15), (0, 18, 3),
                                       (1, 21, 5), (0, 30, 0), (0, 32, 31),
                                       (0, 17, 16), (0, 20, 19), (0, 24, 23), (0, 25, 1),
                                       (0, 28, 27), (0, 29, 3)])   # edges of the 20-, 24- and 28-entry rows
def test_phase_link_parity(ctx, cfg, N, ref):
    win = (5, 11, 3, 6) if cfg == 1 else (5, 11, 1, 1)
    C32 = oracle_C(cfg, N, 40, 70, win, seed=21 + N)
    o = oracle.phase_link(C32.astype(np.complex128), N, ref, cond=True)
    g = ctx.phase_link(torch.from_numpy(C32).cuda(), N, ref)
    ph_g, tc_g, st_g = to_np(g["phase"]), to_np(g["tcoh"]), to_np(g["status"])
    live = o["status"] != 3
    assert np.array_equal(st_g == 3, ~live)
    # the eigenvector is unique only with a gap; exclude (and count) degenerate pixels
    clear, n_degenerate = clear_of_degenerate(o, live)
    rep = phase_report(ph_g, o["phase"], clear)
    print(f"N={N}: {n_degenerate} of {int(live.sum())} live pixels degenerate; phase {rep}")
    assert rep["max"] <= PHASE_TOL, rep
    assert np.all(ph_g[ref][live] == 0.0)
    assert np.nanmax(np.abs(tc_g[live] - o["tcoh"][live])) <= TCOH_TOL
    assert n_degenerate <= 0.02 * live.sum()


@pytest.mark.parametrize("cfg,N,ref", [(1, 15, 0), (2, 15, 3)])
def test_phase_link_without_fp64_resolve(plk, ctx, cfg, N, ref):
    # fp64_resolve = 0 keeps every pixel in single precision: no pixel reports
    # the double-precision status, and every pixel the default mode also
    # solves in single precision gets the same answer (same kernel, same path).
    win = (5, 11, 3, 6) if cfg == 1 else (5, 11, 1, 1)
    C32 = oracle_C(cfg, N, 60, 90, win, seed=40 + cfg)
    Cg = torch.from_numpy(C32).cuda()
    d = ctx.phase_link(Cg, N, ref)
    s = ctx.phase_link(Cg, N, ref, plk.default_params(fp64_resolve=0))
    st_d, st_s = to_np(d["status"]), to_np(s["status"])
    assert not np.any(st_s == 1)
    same = st_d == 0
    assert np.array_equal(st_s[same], st_d[same])
    assert np.array_equal(to_np(s["phase"])[:, same], to_np(d["phase"])[:, same])
    o = oracle.phase_link(C32.astype(np.complex128), N, ref)
    clear, _ = clear_of_degenerate(o, same)
    assert phase_report(to_np(s["phase"]), o["phase"], clear)["max"] <= PHASE_TOL
    print(f"workload {cfg}: {np.sum(st_d == 1)} pixels re-solved in double precision by default, "
          f"statuses without: {np.bincount(st_s.ravel(), minlength=5).tolist()}")


# Capacity of the pending list through which the single-precision pass hands
# its flagged pixels to the double-precision re-solve; past it the re-solve
# scans the statuses instead.
PENDING_LIST_CAP = 65536


def test_fp64_resolve_pending_list_and_status_scan(plk, ctx):
    # 96,000 output pixels at N = 5 (3x3 window, stride 1).  cond_max = 1 flags
    # every pixel whose G is invertible (more than the list holds: the re-solve
    # scans the statuses); a cond_max that about 10,000 pixels exceed (by the
    # oracle's 2-norm condition numbers) goes through the list.  Both runs
    # re-solve their pixels in double precision to the oracle's answer, and a
    # pixel re-solved in both gets the same answer bit for bit.
    N, ref = 5, 0
    C32 = oracle_C(0, N, 320, 300, (3, 3, 1, 1), seed=77)
    Cg = torch.from_numpy(C32).cuda()
    o = oracle.phase_link(C32.astype(np.complex128), N, ref, cond=True)
    live = o["status"] != 3
    clear, _ = clear_of_degenerate(o, live)
    cg = o["condG"][live & np.isfinite(o["condG"])]
    cond_list = float(np.quantile(cg, 1.0 - 10000 / cg.size))
    runs = {}
    for name, prm in (("list", plk.default_params(cond_max=cond_list)), ("scan", plk.default_params(cond_max=1.0))):
        g = ctx.phase_link(Cg, N, ref, prm)
        ph, st = to_np(g["phase"]), to_np(g["status"])
        assert np.array_equal(st == 3, ~live)
        rep = phase_report(ph, o["phase"], clear)
        assert rep["max"] <= PHASE_TOL, (name, rep)
        assert np.nanmax(np.abs(to_np(g["tcoh"])[live] - o["tcoh"][live])) <= TCOH_TOL
        runs[name] = (ph, st)
        print(f"{name}: {int(np.sum(st == 1))} pixels re-solved in double precision; phase {rep}")
    n_list, n_scan = int(np.sum(runs["list"][1] == 1)), int(np.sum(runs["scan"][1] == 1))
    assert 0 < n_list <= PENDING_LIST_CAP < n_scan
    both = (runs["list"][1] == 1) & (runs["scan"][1] == 1)
    assert np.array_equal(runs["list"][0][:, both], runs["scan"][0][:, both])


def test_phase_link_closed_forms(ctx):
    # N=2: linked phase = interferogram phase, gamma_t = 1, lambda_min = 1.
    rng = np.random.default_rng(5)
    g = rng.uniform(0.05, 0.95, 1000)
    th = rng.uniform(-np.pi, np.pi, 1000)
    C = np.stack([np.ones(1000), g * np.exp(1j * th), np.ones(1000)], 1).astype(np.complex64)
    out = ctx.phase_link(torch.from_numpy(C).cuda(), 2, 0)
    d = wrapped_diff(to_np(out["phase"])[1], np.angle(np.conj(C[:, 1])))
    assert d.max() < 1e-5
    assert np.abs(to_np(out["tcoh"]) - 1).max() < 1e-6
    assert np.abs(to_np(out["lam"]) - 1).max() < 1e-4


# -------------------------------------------------------------------- S7

@pytest.mark.parametrize("win,first_real,N,W", [((5, 11, 3, 6), 0, 6, 101), ((5, 11, 1, 1), 2, 6, 101),
                                                 ((3, 5, 4, 7), 1, 6, 101), ((5, 11, 3, 6), 1, 13, 600),
                                                 ((5, 11, 1, 1), 0, 11, 530)])
def test_compress_parity(ctx, win, first_real, N, W):
    H = 45
    z, _ = stack(0, N=N, H=H, W=W, seed=31)
    Ho, Wo = H // win[2], W // win[3]
    rng = np.random.default_rng(1)
    ph = rng.uniform(-np.pi, np.pi, (N, Ho, Wo)).astype(np.float32)
    ph[:, 2, 3] = np.nan
    k_o = oracle.compress(z.numpy(), first_real, win, ph.astype(np.float64))
    k_g = to_np(ctx.compress(z.cuda(), first_real, win, torch.from_numpy(ph).cuda()))
    scale = np.abs(z.numpy()[first_real:]).sum(0)
    assert np.max(np.abs(k_g - k_o) / (scale + 1e-6)) < 2e-6


# ------------------------------------------------------------- S1-S8 chain

def chain_case(case):
    if case == "n10_128px":
        z, spec = stack(0, H=72, W=90)
        return z, (5, 11, 1, 1), 10, 6, 10
    if case == "burst_n15":
        z, spec = stack(1, H=96, W=300)
        return z, (5, 11, 3, 6), 15, 6, 15
    z, spec = stack(3, scale=0.05)  # 60 dates, 102 x 205, step patch inside
    return z, (5, 11, 1, 1), 15, 3, 60


@pytest.mark.parametrize("case", ["n10_128px", "burst_n15", "chain_60d"])
def test_ministack_step_parity(plk, ctx, case, tmp_path):
    """Each step from identical inputs: the oracle's state (compressed SLCs as
    stored complex64 samples, power sums) is loaded into the library through its
    checkpoint format, and one step of both is compared."""
    z, window, M, K_max, nd = chain_case(case)
    H, W = z.shape[1:]
    orc = oracle.OracleChain(H, W, window, K_max=K_max, alpha=1e-3, kappa_dtype=np.complex64)
    zg = z.cuda()
    for k, sl in enumerate(synth.ministack_slices(nd, M)):
        path = str(tmp_path / f"s{k}.plk")
        write_state_file(path, orc)
        st = plk.State.load(ctx, path, M_max=M)
        g = st.step(zg[sl].contiguous())
        o = orc.step(z[sl].numpy())
        assert np.array_equal(count_np(g["count"]), o["count"]), k
        live = o["status"] != 3
        assert np.array_equal(to_np(g["status"]) == 3, ~live)
        clear = live & (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
        K = o["K_used"]
        rep = phase_report(to_np(g["phase"]), o["phase"][K:], clear)
        assert rep["max"] <= PHASE_TOL, (k, rep)
        tc = np.abs(to_np(g["tcoh"]) - o["tcoh"])[live]
        assert tc.max() <= TCOH_TOL, (k, tc.max())
        assert clear.sum() >= 0.99 * live.sum()
        # the new compressed SLC
        kg = to_np(st.kappa(st.info()["K_used"] - 1))
        ko = orc.ring[-1]
        scale = np.abs(z[sl].numpy()).sum(0)
        assert np.max(np.abs(kg - ko) / (scale + 1e-6)) < 1e-4
        assert np.array_equal(to_np(st.sum_pow()), orc.sum_pow)
        st.close()


@pytest.mark.parametrize("case", ["burst_n15", "chain_60d"])
def test_ministack_chain_end_to_end(plk, ctx, case):
    """The whole chain, each side carrying its own compressed SLCs: single-
    precision differences in kappa propagate, so the bar is statistical
    (p99 within the phase tolerance) plus exact masks and power sums."""
    z, window, M, K_max, nd = chain_case(case)
    H, W = z.shape[1:]
    st = plk.State(ctx, H, W, window, K_max=K_max, M_max=M)
    orc = oracle.OracleChain(H, W, window, K_max=K_max, alpha=1e-3)
    zg = z.cuda()
    for k, sl in enumerate(synth.ministack_slices(nd, M)):
        g = st.step(zg[sl].contiguous())
        o = orc.step(z[sl].numpy())
        assert np.array_equal(count_np(g["count"]), o["count"]), k
        live = o["status"] != 3
        K = o["K_used"]
        d = wrapped_diff(to_np(g["phase"]), o["phase"][K:])[:, live]
        assert np.percentile(d, 99) <= PHASE_TOL, (k, np.percentile(d, 99))
        assert np.median(d) <= 0.1 * PHASE_TOL
    info = st.info()
    assert info["n_eff"] == nd and info["K_used"] == min(K_max, len(synth.ministack_slices(nd, M)))
    assert np.array_equal(to_np(st.sum_pow()), orc.sum_pow)


def test_chain_checkpoint_resume(plk, ctx, tmp_path):
    z, _ = stack(3, scale=0.03)
    window, M = (5, 11, 1, 1), 15
    H, W = z.shape[1:]
    zg = z.cuda()
    a = plk.State(ctx, H, W, window, K_max=3, M_max=M)
    outs_a = [a.step(zg[sl].contiguous()) for sl in synth.ministack_slices(60, M)]
    b = plk.State(ctx, H, W, window, K_max=3, M_max=M)
    for sl in synth.ministack_slices(60, M)[:2]:
        b.step(zg[sl].contiguous())
    path = str(tmp_path / "chain.plk")
    b.save(path)
    b.close()
    c = plk.State.load(ctx, path, M_max=M)
    outs_c = [c.step(zg[sl].contiguous()) for sl in synth.ministack_slices(60, M)[2:]]
    for ga, gc in zip(outs_a[2:], outs_c):
        assert torch.equal(ga["phase"], gc["phase"])
        assert torch.equal(ga["tcoh"], gc["tcoh"])
    assert c.info() == a.info()


# ------------------------------------------------------------------ edges

def test_edge_cases(plk, ctx):
    # Output grid empty (H < sy): nothing to do, no error.
    z = torch.zeros((3, 2, 50), dtype=torch.complex64, device="cuda")
    st = plk.State(ctx, 2, 50, (5, 11, 3, 6), K_max=2, M_max=3)
    out = st.step(z)
    assert out["phase"].shape == (3, 0, 8)
    # An all-zero image is all no-data.
    st2 = plk.State(ctx, 9, 20, (5, 11, 1, 1), K_max=2, M_max=3)
    out = st2.step(torch.zeros((3, 9, 20), dtype=torch.complex64, device="cuda"))
    assert torch.all(out["status"] == plk.PX_NODATA) and torch.all(torch.isnan(out["phase"]))
    # A window larger than the image, and N = 2.
    zz, _ = stack(0, N=2, H=3, W=4, seed=2)
    st3 = plk.State(ctx, 3, 4, (5, 11, 1, 1), K_max=0, M_max=2)
    g = st3.step(zz.cuda())
    orc = oracle.OracleChain(3, 4, (5, 11, 1, 1), K_max=0)
    o = orc.step(zz.numpy())
    assert np.array_equal(count_np(g["count"]), o["count"])
    assert wrapped_diff(to_np(g["phase"]), o["phase_real"]).max() < PHASE_TOL
    # Bad arguments are rejected before any launch.
    with pytest.raises(plk.PlkError):
        plk.State(ctx, 10, 10, (4, 11, 1, 1), K_max=2, M_max=3)
    with pytest.raises(plk.PlkError):
        plk.State(ctx, 10, 10, (5, 11, 1, 1), K_max=20, M_max=15)
    with pytest.raises(plk.PlkError):
        ctx.phase_link(torch.zeros((4, 3), dtype=torch.complex64, device="cuda"), 2, 5)


@pytest.mark.parametrize("case", ["burst_n15", "chain_60d"])
def test_ministack_step_parity_last_real_scheme(plk, ctx, case, tmp_path):
    """The production reference scheme (each compressed SLC carries its
    mini-stack's last real date): every step from identical inputs against the
    oracle chain in the same scheme."""
    z, window, M, K_max, nd = chain_case(case)
    H, W = z.shape[1:]
    orc = oracle.OracleChain(H, W, window, K_max=K_max, alpha=1e-3, kappa_dtype=np.complex64, scheme="last")
    prm = plk.default_params(ref_scheme=plk.REF_LAST_REAL)
    zg = z.cuda()
    for k, sl in enumerate(synth.ministack_slices(nd, M)):
        path = str(tmp_path / f"s{k}.plk")
        write_state_file(path, orc)
        st = plk.State.load(ctx, path, M_max=M)
        g = st.step(zg[sl].contiguous(), prm)
        o = orc.step(z[sl].numpy())
        live = o["status"] != 3
        clear = live & (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
        rep = phase_report(to_np(g["phase"]), o["phase"][o["K_used"]:], clear)
        assert rep["max"] <= PHASE_TOL, (k, rep)
        kg = to_np(st.kappa(st.info()["K_used"] - 1))
        scale = np.abs(z[sl].numpy()).sum(0)
        assert np.max(np.abs(kg - orc.ring[-1]) / (scale + 1e-6)) < 1e-4
        st.close()


def test_last_real_scheme_noise_free_short_baselines(plk, ctx):
    n_dates, M, H, W = 20, 5, 24, 48
    rng = np.random.default_rng(3)
    t = np.arange(n_dates)
    phi = 0.3 * t + 0.4 * np.sin(t)
    amp = rng.rayleigh(1.0, (H, W)) + 0.2
    psi = rng.uniform(-np.pi, np.pi, (H, W))
    z = torch.from_numpy((amp[None] * np.exp(1j * (phi[:, None, None] + psi[None]))).astype(np.complex64)).cuda()
    st = plk.State(ctx, H, W, (3, 5, 1, 1), K_max=3, M_max=M)
    prm = plk.default_params(ref_scheme=plk.REF_LAST_REAL)
    for s, sl in enumerate(synth.ministack_slices(n_dates, M)):
        g = st.step(z[sl].contiguous(), prm)
        ref_date = 0 if s == 0 else sl.start - 1
        want = (phi[sl] - phi[ref_date])[:, None, None]
        assert wrapped_diff(to_np(g["phase"]), want).max() < 1e-4, s
    st.close()


def _evd_slow_coherences(N, count, seed):
    """Packed coherences (unit diagonal, positive semidefinite) of three
    looks whose |C| is indefinite -- the inversion fails and the EVD fallback
    of Sec. III-B applies -- with lambda_2 / lambda_1 of C above 0.3, so the
    power iteration is slow and the shifted refinement runs."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(N)
    out = []
    while len(out) < count:
        Z = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
        S = Z @ Z.conj().T
        d = 1.0 / np.sqrt(np.real(np.diag(S)))
        C = S * np.outer(d, d)
        if np.linalg.eigvalsh(np.abs(C))[0] > -1e-3:
            continue
        w = np.linalg.eigvalsh(C)
        if w[-2] / w[-1] < 0.35:
            continue
        out.append(C[iu])
    return np.asarray(out).astype(np.complex64)


@pytest.mark.parametrize("N", [8, 12])
def test_evd_fallback_iteration_budget(plk, ctx, N):
    """max_iter caps the EVD fallback's power iteration and its refinement
    together: with a budget of 3 steps the slow pixels report NOCONV (last
    iterate kept, finite phases); with the default budget they converge to the
    oracle's largest eigenvector of C (status EVD, phase within 1e-4 rad)."""
    C = _evd_slow_coherences(N, 64, seed=11)
    o = oracle.phase_link(C.astype(np.complex128), N, 0)
    assert np.all(o["status"] == plk.PX_EVD)
    Cg = torch.from_numpy(C).cuda()
    tight = ctx.phase_link(Cg, N, 0, plk.default_params(max_iter=3, fp64_resolve=0))
    assert np.all(to_np(tight["status"]) == plk.PX_NOCONV)
    assert np.all(np.isfinite(to_np(tight["phase"])))
    full = ctx.phase_link(Cg, N, 0)
    assert np.all(to_np(full["status"]) == plk.PX_EVD)
    assert wrapped_diff(to_np(full["phase"]), o["phase"]).max() <= PHASE_TOL


@pytest.mark.parametrize("win", [(5, 11, 3, 6), (5, 11, 1, 1), (3, 3, 4, 4)])
def test_step_equals_the_separate_calls(plk, ctx, win):
    """plk_ministack_step equals the separate C-ABI calls plk_amp_stats,
    plk_shp_select, plk_estimate_covariance and plk_phase_link on the same
    stack: sums, masks and counts bit for bit, and the same phases, gamma_t and
    statuses, over two steps (the second merges into the running sums).  The
    double-precision re-solve is off on both sides: by design the step
    recomputes a flagged pixel's coherence from the stack, plk_phase_link from
    its single-precision input.  The image size leaves rows and columns outside
    every decimation block."""
    z, _ = stack(1, N=20, H=97, W=301, seed=13)
    zg = z.cuda()
    M = 10
    H, W = z.shape[1:]
    p = plk.default_params(fp64_resolve=0)
    st = plk.State(ctx, H, W, win, K_max=0, M_max=M)
    sp, sa = None, torch.empty((H, W), device="cuda")
    same = lambda a, b: torch.equal(torch.nan_to_num(a, nan=-9.0), torch.nan_to_num(b, nan=-9.0))
    for k, sl in enumerate(synth.ministack_slices(20, M)):
        g = st.step(zg[sl].contiguous(), p)
        sp, sa = ctx.amp_stats(zg[sl].contiguous(), sp, sa, accumulate=k > 0)
        mask, cnt = ctx.shp_select(sp, M * (k + 1), win)
        C = ctx.estimate_covariance(zg[sl].contiguous(), win, mask)
        o = ctx.phase_link(C, M, 0, p)
        assert torch.equal(st.sum_pow(), sp), k
        assert torch.equal(g["count"], cnt), k
        assert torch.equal(g["status"], o["status"]), k
        assert same(g["phase"], o["phase"]) and same(g["tcoh"], o["tcoh"]), k
    st.close()
