"""Parity at the full sizes of the five workloads, in the launch
configurations the bench times, on outputs the FP64 oracle recomputes one by
one from crops of the same inputs (every local input of an output lies in a
crop around it; each crop oracle is checked exact against the whole-image
oracle on small stacks):

- burst (N = 15, 4096 x 16384, 11x5, strides 6x3): sampled output pixels
  (random, corners, double-precision and EVD pixels) and compressed-SLC cells;
- sequential chain (60 dates of 2048 x 4096 in four mini-stacks): sampled
  pixels through every step, the crop holding the dependency cone;
- uneven batch (64 stacks, N = 5..30, recorded graph): sampled pixels;
- adjoint (N = 20, 1024 x 1024): sampled gradient components against central
  differences of the oracle's partial loss;
- the 128 x 128 stack: every pixel.

SHP counts bit-exact, EVD and no-data decisions alike, phase within 1e-4 rad,
gamma_t within 1e-5 (statistical bars for the chain, whose sides carry their
own compressed SLCs).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import GAP_MIN, PHASE_TOL, TCOH_TOL, count_np, to_np, wrapped_diff

pytestmark = pytest.mark.gpu

WINDOW = (5, 11, 3, 6)   # wy, wx, sy, sx
N = 15


@pytest.fixture(scope="module")
def plk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


@pytest.fixture(scope="module")
def burst(plk):
    ctx = plk.Context("cuda:0")
    spec = synth.config_spec(1)
    z = synth.generate(spec, device="cuda")
    st = plk.State(ctx, spec.H, spec.W, WINDOW, K_max=6, M_max=N)
    out = st.step(z)
    torch.cuda.synchronize()
    res = {"z": z, "H": spec.H, "W": spec.W, "phase": to_np(out["phase"]), "tcoh": to_np(out["tcoh"]),
           "status": to_np(out["status"]), "count": count_np(out["count"]),
           "kappa": st.kappa(st.info()["K_used"] - 1)}
    yield res
    res.clear()
    st.close()
    del z, out
    torch.cuda.empty_cache()


def oracle_pixel(b, oy, ox):
    """Oracle phase linking of output pixel (oy, ox) from a crop holding its window."""
    wy, wx, sy, sx = WINDOW
    hy, hx = wy // 2, wx // 2
    cy, cx = oy * sy + sy // 2, ox * sx + sx // 2
    y0, y1 = max(0, cy - hy), min(b["H"], cy + hy + 1)
    x0, x1 = max(0, cx - hx), min(b["W"], cx + hx + 1)
    crop = b["z"][:, y0:y1, x0:x1].cpu().numpy()
    win1 = (wy, wx, 1, 1)   # stride 1 on the crop: output (i, j) is centred on crop pixel (i, j)
    P, _ = oracle.amp_stats(crop)
    m, cnt = oracle.shp_select(P, win1, np.float32(oracle.glrt_threshold(1e-3, N)))
    C = oracle.covariance(crop, win1, m)[cy - y0, cx - x0]
    o = oracle.phase_link(C[None], N, 0)
    return {"count": int(cnt[cy - y0, cx - x0]), "phase": o["phase"][:, 0], "tcoh": o["tcoh"][0],
            "status": int(o["status"][0]), "gap": o["gap"][0], "lam": o["lam"][0]}


def test_sampled_output_pixels_at_full_size(burst):
    Ho, Wo = burst["status"].shape
    assert (Ho, Wo) == (4096 // 3, 16384 // 6)
    rng = np.random.default_rng(2511)
    st = burst["status"]
    pix = [(0, 0), (0, Wo - 1), (Ho - 1, 0), (Ho - 1, Wo - 1)]
    pix += [(int(rng.integers(Ho)), int(rng.integers(Wo))) for _ in range(160)]
    for code in (1, 2):   # double-precision re-solve, EVD fallback
        ys, xs = np.nonzero(st == code)
        pick = rng.choice(ys.size, size=min(40, ys.size), replace=False)
        pix += [(int(ys[i]), int(xs[i])) for i in pick]
    worst, n_clear, kinds = 0.0, 0, {0: 0, 1: 0, 2: 0, 3: 0, 4: 0}
    for oy, ox in pix:
        o = oracle_pixel(burst, oy, ox)
        g_status = int(st[oy, ox])
        kinds[g_status] += 1
        assert burst["count"][oy, ox] == o["count"], (oy, ox)
        if o["status"] == 3:
            assert g_status == 3, (oy, ox)
            continue
        if g_status == 4:        # not converged: no unique answer to compare
            continue
        assert (g_status == 2) == (o["status"] == 2), (oy, ox, g_status, o["status"])
        if o["gap"] > GAP_MIN * abs(o["lam"] if np.isfinite(o["lam"]) else 1.0):
            d = wrapped_diff(burst["phase"][:, oy, ox], o["phase"]).max()
            worst = max(worst, d)
            n_clear += 1
            assert d <= PHASE_TOL, (oy, ox, d)
        assert abs(burst["tcoh"][oy, ox] - o["tcoh"]) <= TCOH_TOL, (oy, ox)
    print(f"full size: {len(pix)} sampled pixels {kinds}, {n_clear} compared, max phase error {worst:.2e} rad")
    assert n_clear >= 0.9 * len(pix)


def test_sampled_compressed_slc_at_full_size(burst):
    wy, wx, sy, sx = WINDOW
    Ho, Wo = burst["status"].shape
    rng = np.random.default_rng(7)
    kg = burst["kappa"]
    for _ in range(40):
        oy, ox = int(rng.integers(Ho)), int(rng.integers(Wo))
        o = oracle_pixel(burst, oy, ox)
        if o["status"] == 3 or burst["status"][oy, ox] == 4 or \
                not o["gap"] > 1e-6 * abs(o["lam"] if np.isfinite(o["lam"]) else 1.0):
            continue
        cell = burst["z"][:, oy * sy:(oy + 1) * sy, ox * sx:(ox + 1) * sx].cpu().numpy()
        ko = oracle.compress(cell, 0, WINDOW, o["phase"].reshape(N, 1, 1))
        kc = to_np(kg[oy * sy:(oy + 1) * sy, ox * sx:(ox + 1) * sx])
        scale = np.abs(cell).sum(0)
        assert np.max(np.abs(kc - ko) / (scale + 1e-6)) < 1e-4, (oy, ox)


# ------------------------------------------------ sequential chain, full size

CHAIN_WINDOW = (5, 11, 1, 1)
CHAIN_K_MAX, CHAIN_M = 3, 15


@pytest.fixture(scope="module")
def chain(plk):
    """Four mini-stack steps of the 60-date 2048 x 4096 chain (a +2 rad step
    from date 31 on a 200 x 200 patch), outputs kept at sampled pixels."""
    ctx = plk.Context("cuda:0")
    spec = synth.config_spec(3)
    z = synth.generate(spec, device="cuda")
    H, W = spec.H, spec.W
    rng = np.random.default_rng(60)
    pix = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0)]
    pix += [(int(rng.integers(H)), int(rng.integers(W))) for _ in range(40)]
    pix += [(int(rng.integers(924, 1124)), int(rng.integers(1948, 2148))) for _ in range(16)]   # the step patch
    ys = torch.tensor([p[0] for p in pix], device="cuda")
    xs = torch.tensor([p[1] for p in pix], device="cuda")
    st = plk.State(ctx, H, W, CHAIN_WINDOW, K_max=CHAIN_K_MAX, M_max=CHAIN_M)
    steps = []
    for sl in synth.ministack_slices(spec.N, CHAIN_M):
        g = st.step(z[sl].contiguous())
        steps.append({"phase": to_np(g["phase"][:, ys, xs]), "tcoh": to_np(g["tcoh"][ys, xs]),
                      "status": to_np(g["status"][ys, xs]), "count": count_np(g["count"][ys, xs])})
    kap = [to_np(st.kappa(i)[ys, xs]) for i in range(st.info()["K_used"])]
    yield {"z": z, "H": H, "W": W, "N": spec.N, "pix": pix, "steps": steps, "kappa": kap}
    st.close()
    del z
    torch.cuda.empty_cache()


def test_chain_sampled_at_full_size(chain):
    # An output of step k reaches back through the compressed SLCs of the
    # earlier steps, each a window further: after four steps, 4 * 2 rows and
    # 4 * 5 columns.  The oracle runs the whole chain on a crop with that
    # margin (and two more) around each sampled pixel.
    wy, wx, _, _ = CHAIN_WINDOW
    my, mx = 4 * (wy // 2) + 2, 4 * (wx // 2) + 2
    H, W, Nd = chain["H"], chain["W"], chain["N"]
    diffs, tcd = [], []
    for j, (py, px) in enumerate(chain["pix"]):
        y0, y1 = max(0, py - my), min(H, py + my + 1)
        x0, x1 = max(0, px - mx), min(W, px + mx + 1)
        crop = chain["z"][:, y0:y1, x0:x1].cpu().numpy()
        orc = oracle.OracleChain(y1 - y0, x1 - x0, CHAIN_WINDOW, K_max=CHAIN_K_MAX, alpha=1e-3)
        ly, lx = py - y0, px - x0
        for k, sl in enumerate(synth.ministack_slices(Nd, CHAIN_M)):
            o = orc.step(crop[sl])
            g = chain["steps"][k]
            assert g["count"][j] == o["count"][ly, lx], (j, k)
            if o["status"][ly, lx] == 3:
                assert g["status"][j] == 3
                continue
            K = o["K_used"]
            diffs.append(wrapped_diff(g["phase"][:, j], o["phase"][K:, ly, lx]).max())
            tcd.append(abs(g["tcoh"][j] - o["tcoh"][ly, lx]))
        for i, ko in enumerate(orc.ring):
            scale = np.abs(crop[:, ly, lx]).sum()
            assert abs(chain["kappa"][i][j] - ko[ly, lx]) <= 1e-3 * scale, (j, i)
    diffs, tcd = np.array(diffs), np.array(tcd)
    print(f"chain at full size: {len(chain['pix'])} pixels x 4 steps, phase max {diffs.max():.2e} "
          f"p99 {np.percentile(diffs, 99):.2e} median {np.median(diffs):.2e} rad, gamma_t max {tcd.max():.2e}")
    # each side carries its own compressed SLCs, so the bar is the chain's statistical one
    assert np.percentile(diffs, 99) <= PHASE_TOL
    assert np.median(diffs) <= 0.1 * PHASE_TOL
    assert np.percentile(tcd, 99) <= TCOH_TOL


# ------------------------------------------------- uneven batch, full size

def test_batch_sampled_at_full_size(plk):
    # The batch workload as timed: 64 stacks of 1024 x 2048, N from 5..30,
    # gamma0 from 0.3..0.9, 1% near-singular patches, one recorded graph.
    from paper_2511_12051_gb300 import dist as pdist
    ctx = plk.Context("cuda:0")
    rng = np.random.default_rng(pdist.unit_seed(2, 0))
    Ns = rng.integers(5, 31, 64)
    g0 = rng.uniform(0.3, 0.9, 64)
    zs = [synth.generate(synth.config_spec(2, N=int(Ns[i]), rho0=float(g0[i]), seed=int(rng.integers(1 << 30)),
                                           H=1024, W=2048), device="cuda") for i in range(64)]
    b = plk.Batch(ctx, zs, WINDOW)
    b.run()          # tunes and records
    out = b.run()    # the recorded graph
    torch.cuda.synchronize()
    srng = np.random.default_rng(5)
    diffs, n_fp64, n_evd = [], 0, 0
    for i, (z, o_g) in enumerate(zip(zs, out)):
        st = to_np(o_g["status"])
        Ho, Wo = st.shape
        pix = [(int(srng.integers(Ho)), int(srng.integers(Wo))) for _ in range(3)]
        for code in (1, 2):
            ys, xs = np.nonzero(st == code)
            if ys.size:
                j = int(srng.integers(ys.size))
                pix.append((int(ys[j]), int(xs[j])))
        ph, tc = to_np(o_g["phase"]), to_np(o_g["tcoh"])
        bdict = {"z": z, "H": 1024, "W": 2048}
        for oy, ox in pix:
            o = oracle_pixel_n(bdict, oy, ox, int(Ns[i]))
            assert (o["status"] == 3) == (st[oy, ox] == 3), (i, oy, ox)   # the batch reports no SHP counts
            if o["status"] == 3 or st[oy, ox] == 4:
                continue
            assert (st[oy, ox] == 2) == (o["status"] == 2), (i, oy, ox)
            n_fp64 += int(st[oy, ox] == 1)
            n_evd += int(st[oy, ox] == 2)
            if o["gap"] > GAP_MIN * abs(o["lam"] if np.isfinite(o["lam"]) else 1.0):
                d = wrapped_diff(ph[:, oy, ox], o["phase"]).max()
                diffs.append(d)
                assert d <= PHASE_TOL, (i, oy, ox, d)
            assert abs(tc[oy, ox] - o["tcoh"]) <= TCOH_TOL, (i, oy, ox)
    print(f"batch at full size: {len(diffs)} pixels compared over 64 stacks ({n_fp64} double-precision, "
          f"{n_evd} EVD), max phase error {max(diffs):.2e} rad")
    assert len(diffs) >= 64 * 3
    b.close()
    del zs
    torch.cuda.empty_cache()


def oracle_pixel_n(b, oy, ox, n):
    """oracle_pixel for a stack of n dates (reference date 0)."""
    wy, wx, sy, sx = WINDOW
    hy, hx = wy // 2, wx // 2
    cy, cx = oy * sy + sy // 2, ox * sx + sx // 2
    y0, y1 = max(0, cy - hy), min(b["H"], cy + hy + 1)
    x0, x1 = max(0, cx - hx), min(b["W"], cx + hx + 1)
    crop = b["z"][:, y0:y1, x0:x1].cpu().numpy()
    win1 = (wy, wx, 1, 1)
    P, _ = oracle.amp_stats(crop)
    m, cnt = oracle.shp_select(P, win1, np.float32(oracle.glrt_threshold(1e-3, n)))
    C = oracle.covariance(crop, win1, m)[cy - y0, cx - x0]
    o = oracle.phase_link(C[None], n, 0)
    return {"count": int(cnt[cy - y0, cx - x0]), "phase": o["phase"][:, 0], "tcoh": o["tcoh"][0],
            "status": int(o["status"][0]), "gap": o["gap"][0], "lam": o["lam"][0]}


# ------------------------------------------------------ adjoint, full size

def test_adjoint_sampled_at_full_size(plk):
    # The adjoint workload as timed: N = 20 x 1024 x 1024, 11x5 window, stride
    # 1, masks frozen, L = sum(w * phase), w ~ U(-1, 1).  The gradient at a
    # sample q sums over the output pixels whose windows hold q (rows q +- 2,
    # columns q +- 5), each depending on its own window: a crop of q +- 4 rows
    # and +- 10 columns (plus 1) holds all of it.  Oracle: central differences
    # (h = 1e-6) of that partial loss, with the crop's own oracle SHP masks
    # (checked equal to the library's); the weights of pixels the oracle finds
    # near the wrap or off the EMI path are set to 0 on both sides.
    ctx = plk.Context("cuda:0")
    win = (5, 11, 1, 1)
    spec = synth.config_spec(4)
    z = synth.generate(spec, device="cuda")
    Nd, H, W = z.shape
    P, _ = ctx.amp_stats(z)
    mask, _ = ctx.shp_select(P, Nd, win, 1e-3)
    g = torch.Generator(device="cuda").manual_seed(4)
    wn = to_np(torch.rand((Nd, H, W), device="cuda", generator=g) * 2 - 1)
    srng = np.random.default_rng(20)
    qs = [(int(srng.integers(H)), int(srng.integers(W))) for _ in range(12)] + [(0, 0), (H - 1, W - 1)]
    nb = win[0] * win[1]
    thr = np.float32(oracle.glrt_threshold(1e-3, Nd))
    mk = to_np(mask).view(np.uint64)
    cases = []
    for (qy, qx) in qs:
        y0, y1 = max(0, qy - 5), min(H, qy + 6)
        x0, x1 = max(0, qx - 11), min(W, qx + 12)
        crop = z[:, y0:y1, x0:x1].cpu().numpy().astype(np.complex128)
        Pc, _ = oracle.amp_stats(crop.astype(np.complex64))
        mc, _ = oracle.shp_select(Pc, win, thr)   # stride 1: crop pixel (i, j) is output (i, j)
        py0, py1 = max(0, qy - 2), min(H, qy + 3)   # output pixels whose windows hold q
        px0, px1 = max(0, qx - 5), min(W, qx + 6)
        for py in range(py0, py1):
            for px in range(px0, px1):
                assert np.array_equal(mk[py, px], mc[py - y0, px - x0]), (py, px)
                s, _ = oracle.window_samples(crop, win, py - y0, px - x0)   # all in-image samples are in the crop
                o = oracle.phase_link(oracle.weighted_coherence(s, oracle.mask_weights(mc[py - y0, px - x0], nb))[None],
                                      Nd, 0)
                if o["status"][0] != 0 or np.any(np.abs(o["phase"][:, 0]) > np.pi - 0.05):
                    wn[:, py, px] = 0.0          # ill-posed: no weight on either side
        cases.append((qy, qx, y0, x0, py0, py1, px0, px1, crop, mc))
    grad = to_np(ctx.phase_link_backward(z, win, mask, 0, torch.from_numpy(wn).cuda(),
                                         plk.default_params(fp64_resolve=0)))
    errs, refs = [], []
    h = 1e-6
    for (qy, qx, y0, x0, py0, py1, px0, px1, crop, mc) in cases:
        def loss(zc):
            tot = 0.0
            for py in range(py0, py1):
                for px in range(px0, px1):
                    if not np.any(wn[:, py, px]):
                        continue
                    s, _ = oracle.window_samples(zc, win, py - y0, px - x0)
                    Cw = oracle.weighted_coherence(s, oracle.mask_weights(mc[py - y0, px - x0], nb))
                    tot += float(np.dot(wn[:, py, px], oracle.phase_link(Cw[None], Nd, 0)["phase"][:, 0]))
            return tot

        ly, lx = qy - y0, qx - x0
        for i in srng.choice(Nd, size=2, replace=False):
            for comp in (1.0, 1j):
                zp, zm = crop.copy(), crop.copy()
                zp[i, ly, lx] += h * comp
                zm[i, ly, lx] -= h * comp
                fd = (loss(zp) - loss(zm)) / (2 * h)
                ad = grad[i, qy, qx].real if comp == 1.0 else grad[i, qy, qx].imag
                errs.append(abs(ad - fd))
                refs.append(abs(fd))
    errs, refs = np.array(errs), np.array(refs)
    print(f"adjoint at full size: {errs.size} gradient components, max abs err {errs.max():.2e}, "
          f"max |grad| {refs.max():.2e}")
    assert np.all(errs <= 1e-3 * max(refs.max(), 1e-6) + 5e-3 * refs)
    del z
    torch.cuda.empty_cache()


# ------------------------------------------------ 128 x 128 stack, every pixel

def test_small_stack_every_pixel(plk):
    # N = 10 x 128 x 128, 11x5 window, stride 1, GLRT at alpha = 1e-3: the
    # whole image through one step against the whole-image oracle.
    ctx = plk.Context("cuda:0")
    win = (5, 11, 1, 1)
    z = synth.generate(synth.config_spec(0))
    Nd, H, W = z.shape
    assert (Nd, H, W) == (10, 128, 128)
    st = plk.State(ctx, H, W, win, K_max=6, M_max=Nd)
    g = st.step(z.cuda())
    orc = oracle.OracleChain(H, W, win, K_max=6, alpha=1e-3, kappa_dtype=np.complex64)
    o = orc.step(z.numpy())
    assert np.array_equal(count_np(g["count"]), o["count"])
    live = o["status"] != 3
    assert np.array_equal(to_np(g["status"]) == 3, ~live)
    clear = live & (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0)))
    assert clear.sum() >= 0.99 * live.sum()
    d = wrapped_diff(to_np(g["phase"]), o["phase"][o["K_used"]:])[:, clear]
    assert d.max() <= PHASE_TOL, d.max()
    assert np.abs(to_np(g["tcoh"]) - o["tcoh"])[live].max() <= TCOH_TOL
    kg = to_np(st.kappa(st.info()["K_used"] - 1))
    assert np.max(np.abs(kg - orc.ring[-1]) / (np.abs(z.numpy()).sum(0) + 1e-6)) < 1e-4
    print(f"128x128: {clear.sum()} of {live.sum()} pixels compared, max phase error {d.max():.2e} rad")
    st.close()
