"""Spatial tiles (plk_tile_plan): the plan's geometry, and the oracle chain run
tile by tile on the planned crops reproducing, on every tile's owned cells and
pixels, the oracle chain run on the whole burst, bit for bit, at every step.
The oracle is the arbiter here because the claim is about the method's
dependency structure (windows and the compressed SLCs along the chain), not
about a kernel."""
import numpy as np
import pytest

import oracle
from paper_2511_12051_gb300 import dist as pdist
from paper_2511_12051_gb300 import synth


@pytest.fixture(scope="module")
def plk():
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


@pytest.mark.parametrize("H,W,win,ty,tx,steps", [
    (36, 60, (5, 11, 1, 1), 2, 3, 1), (36, 60, (5, 11, 1, 1), 3, 2, 4), (100, 131, (5, 11, 3, 6), 4, 3, 2),
    (61, 97, (19, 37, 3, 6), 2, 2, 3), (20, 20, (1, 1, 1, 1), 5, 4, 2), (47, 53, (3, 3, 2, 2), 23, 26, 1)])
def test_plan_partitions_the_burst(plk, H, W, win, ty, tx, steps):
    wy, wx, sy, sx = win
    Ho, Wo = H // sy, W // sx
    tiles = plk.tile_plan(H, W, win, ty, tx, steps)
    assert len(tiles) == ty * tx
    cells = np.zeros((Ho, Wo), np.int32)
    pixels = np.zeros((H, W), np.int32)
    for t in tiles:
        assert t["y0"] % sy == 0 and t["x0"] % sx == 0
        assert 0 <= t["y0"] and t["y0"] + t["h"] <= H and 0 <= t["x0"] and t["x0"] + t["w"] <= W
        # owned cells are cells of the crop's grid, at the stated offset
        assert t["cy0"] == t["oy0"] - t["y0"] // sy and t["cx0"] == t["ox0"] - t["x0"] // sx
        assert t["cy0"] >= 0 and t["cy0"] + t["oh"] <= t["h"] // sy
        assert t["cx0"] >= 0 and t["cx0"] + t["ow"] <= t["w"] // sx
        # every owned cell's window (clipped to the burst) lies in the crop
        for i in (t["oy0"], t["oy0"] + t["oh"] - 1):
            c = i * sy + sy // 2
            assert max(0, c - wy // 2) >= t["y0"] and min(H, c + wy // 2 + 1) <= t["y0"] + t["h"]
        for j in (t["ox0"], t["ox0"] + t["ow"] - 1):
            c = j * sx + sx // 2
            assert max(0, c - wx // 2) >= t["x0"] and min(W, c + wx // 2 + 1) <= t["x0"] + t["w"]
        cells[t["oy0"]:t["oy0"] + t["oh"], t["ox0"]:t["ox0"] + t["ow"]] += 1
        pixels[t["py0"]:t["py0"] + t["ph"], t["px0"]:t["px0"] + t["pw"]] += 1
        assert t["py0"] == t["oy0"] * sy and t["px0"] == t["ox0"] * sx
    assert np.all(cells == 1) and np.all(pixels == 1)


def test_plan_halo_grows_one_window_a_step(plk):
    # stride 1: the crop reaches hy (hx) beyond the owned cells per step
    H, W, win = 64, 96, (5, 11, 1, 1)
    for steps in (1, 2, 5):
        t = plk.tile_plan(H, W, win, 2, 2, steps)[3]  # the bottom-right tile
        assert (t["y0"], t["x0"]) == (32 - 2 * steps, 48 - 5 * steps)
        assert (t["h"], t["w"]) == (32 + 2 * steps, 48 + 5 * steps)


def test_plan_rejects_bad_requests(plk):
    for args in [(10, 10, (3, 3, 1, 1), 11, 1, 1), (10, 10, (3, 3, 1, 1), 1, 1, 0), (10, 10, (4, 3, 1, 1), 1, 1, 1),
                 (10, 10, (3, 3, 1, 1), 1, 1, 257),
                 (10, 10, (3, 3, 1, 1), 0, 1, 1), (5, 10, (3, 3, 6, 1), 1, 1, 1)]:
        with pytest.raises(plk.PlkError):
            plk.tile_plan(*args)


def _run_chain(z, window, K_max, M, **kw):
    """Oracle chain over z [T, h, w] in mini-stacks of M; the outputs of every step."""
    ch = oracle.OracleChain(z.shape[1], z.shape[2], window, K_max=K_max, kappa_dtype=np.complex64, **kw)
    outs = []
    for sl in synth.ministack_slices(z.shape[0], M):
        o = ch.step(z[sl])
        outs.append({"phase": o["phase_real"], "tcoh": o["tcoh"], "status": o["status"], "count": o["count"],
                     "kappa": ch.ring[-1]})
    return outs


def _owned_equal(whole, part, t):
    sl = pdist.tile_slices(t)
    for k in ("phase", "tcoh", "status", "count"):
        if not np.array_equal(whole[k][(Ellipsis,) + sl["burst_cells"]], part[k][(Ellipsis,) + sl["cells"]],
                              equal_nan=True):
            return False
    return np.array_equal(whole["kappa"][sl["burst_pixels"]], part["kappa"][sl["pixels"]])


@pytest.mark.parametrize("cfg,H,W,win,ty,tx,T,M,K_max,kw", [
    (0, 36, 60, (5, 11, 1, 1), 2, 3, 30, 10, 3, {}),
    (1, 60, 96, (5, 11, 3, 6), 2, 2, 30, 10, 2, {}),
    (1, 60, 96, (5, 11, 3, 6), 3, 2, 20, 10, 3, {"scheme": "last"}),
    (1, 62, 99, (5, 11, 3, 6), 2, 2, 20, 10, 3, {"ps_da_max": 0.2}),
])
def test_tiles_reproduce_the_whole_burst(plk, cfg, H, W, win, ty, tx, T, M, K_max, kw):
    z = synth.generate(synth.config_spec(cfg, N=T, H=H, W=W, seed=91)).numpy()
    steps = len(synth.ministack_slices(T, M))
    whole = _run_chain(z, win, K_max, M, **kw)
    for t in plk.tile_plan(H, W, win, ty, tx, steps):
        crop = np.ascontiguousarray(z[(slice(None),) + pdist.tile_slices(t)["crop"]])
        part = _run_chain(crop, win, K_max, M, **kw)
        for s in range(steps):
            assert _owned_equal(whole[s], part[s], t), (t, s)


def test_a_one_step_halo_is_too_small_for_a_chain(plk):
    # planted mistake: crops planned for one step, run for three -- the
    # compressed SLCs at the crop edges come from truncated windows and reach
    # the owned cells at the next step
    H, W, win, T, M = 36, 60, (5, 11, 1, 1), 30, 10
    z = synth.generate(synth.config_spec(0, N=T, H=H, W=W, seed=91)).numpy()
    whole = _run_chain(z, win, 3, M)
    differs = []
    for t in plk.tile_plan(H, W, win, 2, 2, 1):
        crop = np.ascontiguousarray(z[(slice(None),) + pdist.tile_slices(t)["crop"]])
        part = _run_chain(crop, win, 3, M)
        assert _owned_equal(whole[0], part[0], t)
        differs.append(not _owned_equal(whole[2], part[2], t))
    assert any(differs)
