"""Spatial tiles on the GPU path: every tile of a plk_tile_plan run as its own
state on its crop gives, on its owned cells and pixels, exactly the library's
whole-burst results at every step of the chain (the per-pixel arithmetic does
not depend on where a pixel sits in the image or in a CTA tile).  The
whole-burst results themselves are held to the oracle by the parity tests."""
import numpy as np
import pytest
import torch

from paper_2511_12051_gb300 import dist as pdist
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


def _chain(plk, ctx, z, win, K_max, M, params):
    st = plk.State(ctx, z.shape[1], z.shape[2], win, K_max=K_max, M_max=M)
    outs = []
    for sl in synth.ministack_slices(z.shape[0], M):
        g = st.step(z[sl].contiguous(), params)
        outs.append({k: to_np(g[k]) for k in ("phase", "tcoh", "status")} |
                    {"count": to_np(g["count"]).view(np.uint16), "kappa": to_np(st.kappa(st.info()["K_used"] - 1))})
    st.close()
    return outs


@pytest.mark.parametrize("cfg,H,W,win,tiles,T,M,K_max,over", [
    (0, 192, 320, (5, 11, 1, 1), (2, 3), 30, 10, 3, {}),
    (1, 600, 1200, (5, 11, 3, 6), (3, 2), 30, 15, 2, {}),
    (1, 600, 1200, (5, 11, 3, 6), (2, 2), 30, 15, 2, {"ps_da_max": 0.2}),
    (1, 600, 1200, (5, 11, 3, 6), (2, 2), 30, 15, 2, {"ref_scheme": 1}),
])
def test_tiles_equal_the_whole_burst(plk, ctx, cfg, H, W, win, tiles, T, M, K_max, over):
    z = synth.generate(synth.config_spec(cfg, N=T, H=H, W=W, seed=13)).cuda()
    params = plk.default_params(**over)
    steps = len(synth.ministack_slices(T, M))
    whole = _chain(plk, ctx, z, win, K_max, M, params)
    for t in plk.tile_plan(H, W, win, *tiles, steps):
        sl = pdist.tile_slices(t)
        part = _chain(plk, ctx, z[(slice(None),) + sl["crop"]].contiguous(), win, K_max, M, params)
        for s in range(steps):
            for k in ("phase", "tcoh", "status", "count"):
                a = whole[s][k][(Ellipsis,) + sl["burst_cells"]]
                b = part[s][k][(Ellipsis,) + sl["cells"]]
                assert np.array_equal(a, b, equal_nan=True), (t, s, k)
            assert np.array_equal(whole[s]["kappa"][sl["burst_pixels"]], part[s]["kappa"][sl["pixels"]]), (t, s)
