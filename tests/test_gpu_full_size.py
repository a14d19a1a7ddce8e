"""Parity at the full burst size, in the launch configuration the bench times.

One mini-stack step on the burst-shaped workload (N = 15 complex64 SLCs of
4096 x 16384 pixels, 11x5 window, output strides 6x3, default parameters, a
state with room for 6 compressed SLCs and 15 new ones), then sampled outputs
recomputed one by one by the FP64 oracle from crops of the same stack:

- output pixels (random, the four corners, and pixels the library sent to the
  EVD fallback or the double-precision re-solve): SHP count bit-exact, no-data
  and EVD decisions alike, phase within 1e-4 rad, gamma_t within 1e-5;
- output cells: the compressed SLC at their 3 x 6 full-resolution pixels.

Every local quantity the oracle needs lies inside a crop around the pixel:
the amplitude sums are per pixel, and the SHP test, the coherence and the
compression only reach the pixel's window or cell.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import PHASE_TOL, TCOH_TOL, count_np, to_np, wrapped_diff

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
        if o["gap"] > 1e-6 * abs(o["lam"] if np.isfinite(o["lam"]) else 1.0):
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
