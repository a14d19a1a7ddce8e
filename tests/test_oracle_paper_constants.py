"""Pins from values the paper prints (tests/golden/paper_constants.json)."""
import json
import os

import numpy as np

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_window_table_axis_convention():
    # Full window = 2h + 1 per axis, listed X (columns) first: a window "X x Y"
    # has wx = X columns and wy = Y rows.  The SHP mask of a constant scene
    # must then span exactly X columns and Y rows.
    for row in GOLD["shp_windows_half_x_y_full_X_Y"]["rows"]:
        (hx, hy), (X, Y) = row["half"], row["full"]
        assert (2 * hx + 1, 2 * hy + 1) == (X, Y)
        H, W = 2 * Y + 1, 2 * X + 1
        P = np.ones((H, W), np.float32)
        mask, count = oracle.shp_select(P, (Y, X, 1, 1), np.float32(2.0))
        assert mask.shape[-1] == (X * Y + 63) // 64
        assert count[Y, X] == X * Y


def test_gamma_t_two_images_is_one():
    C = np.array([1.0, 0.42 * np.exp(-1.3j), 1.0])
    assert abs(oracle.temporal_coherence(C, np.array([0.0, 0.77])) - GOLD["gamma_t_for_two_images"]["value"]) < 1e-15


def test_decimation_block_size():
    sx, sy = GOLD["output_strides_x_y"]["value"]
    assert sx * sy == GOLD["decimation_speedup"]["value"]
