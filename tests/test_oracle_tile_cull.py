"""Pins of the oracle's camera tile cull (tile-extent option 4).

A pair (tile, Gaussian) of the 3-sigma box is not listed when alpha cannot reach 1/255 at
any pixel of the tile at that pixel's row time.  The oracle decides it by the minimum of
the Mahalanobis form over the tile's pixel-centre rectangle grown by the mean's sweep; the
pins check that minimum against brute-force sampling of the rectangle, check that the
tile's actual pixels never come closer (so the cull is conservative), and check the
consequences: every culled pair blends nowhere in its tile, the lists shrink to a subset in
the same order, and every render stays exactly the same.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2411_16816_gb300 import scenes
from tests.helpers import front_camera

A_MIN = 1.0 / 255.0


def _moving_scene(seed=3, n=600):
    rng = np.random.default_rng(seed)
    g = scenes.random_gaussians(n, seed, lo=(4, -6, -4), hi=(20, 6, 4), log_scale_mu=-1.6, log_scale_sd=0.6,
                                channels=3, dynamic_frac=0.3, vel_sd=3.0)
    cam = front_camera(width=160, height=120, f=110.0, rs_time=0.03, time_offset=0.004,
                       lin_vel=np.array([0.5, -0.2, 12.0]), ang_vel=np.array([0.02, 0.04, -0.03]))
    return g, cam


def _cull(s):
    return dataclasses.replace(s, support=4)


def _pairs(proj, s):
    """All (tile, Gaussian) pairs of the visible Gaussians' 3-sigma boxes."""
    tx_n = -(-s.width // s.tile_w)
    out_t, out_i = [], []
    for i in np.nonzero(proj["visible"])[0]:
        x0, y0, x1, y1 = proj["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                out_t.append(ty * tx_n + tx)
                out_i.append(i)
    return np.array(out_t), np.array(out_i)


def _tile_pixels(s, tile):
    tx_n = -(-s.width // s.tile_w)
    ty, tx = divmod(int(tile), tx_n)
    cols = np.arange(tx * s.tile_w, min(tx * s.tile_w + s.tile_w, s.width)) + 0.5
    rows = np.arange(ty * s.tile_h, min(ty * s.tile_h + s.tile_h, s.height)) + 0.5
    return cols, rows


def _form(rec, du, dv):
    a, b, c = rec[2], rec[3], rec[4]
    return a * du * du + 2 * b * du * dv + c * dv * dv


def test_margin_is_the_minimum_over_the_swept_rectangle():
    g, cam = _moving_scene()
    s = _cull(cam)
    proj = oracle.project(g, s)
    tiles, ids = _pairs(proj, s)
    rng = np.random.default_rng(0)
    pick = rng.choice(len(tiles), 150, replace=False)
    marg = oracle.tile_margin(g, s, tiles[pick], ids[pick], proj)
    H, rs, dt = cam.height, float(np.float32(cam.rs_time)), float(np.float32(cam.time_offset))
    for t, i, m in zip(tiles[pick], ids[pick], marg):
        rec = proj["rec"][i]
        cols, rows = _tile_pixels(cam, t)
        times = (rows / H - 0.5) * rs + dt
        t0, t1 = times[0], times[-1]
        tm, ht = 0.5 * (t0 + t1), 0.5 * abs(t1 - t0)
        cx, cy = rec[0] + rec[7] * tm, rec[1] + rec[8] * tm
        gx, gy = abs(rec[7]) * ht + 2e-3, abs(rec[8]) * ht + 2e-3
        thr = 2 * math.log(255 * rec[5]) * (1 + 2e-3) + 2e-3
        # dense samples of the grown rectangle: never below the exact minimum, and close to it
        u = np.linspace(cols[0] - gx, cols[-1] + gx, 401) - cx
        v = np.linspace(rows[0] - gy, rows[-1] + gy, 401) - cy
        grid = _form(rec, u[:, None], v[None, :]).min()
        exact = m + thr
        assert exact <= grid + 1e-9
        assert grid - exact <= 2e-3 * (1 + exact)
        # the tile's pixels, each at its own row time, see the mean inside the rectangle
        du = cols[None, :] - (rec[0] + rec[7] * times[:, None])
        dv = rows[:, None] - (rec[1] + rec[8] * times[:, None])
        assert _form(rec, du, dv).min() >= exact - 1e-9


def test_every_culled_pair_blends_nowhere_in_its_tile():
    g, cam = _moving_scene(seed=5)
    s = _cull(cam)
    proj = oracle.project(g, s)
    tiles, ids = _pairs(proj, s)
    marg = oracle.tile_margin(g, s, tiles, ids, proj)
    culled = marg > 0
    assert 0.1 < culled.mean() < 0.9
    H, rs, dt = cam.height, float(np.float32(cam.rs_time)), float(np.float32(cam.time_offset))
    for t, i in zip(tiles[culled], ids[culled]):
        rec = proj["rec"][i]
        cols, rows = _tile_pixels(cam, t)
        times = (rows / H - 0.5) * rs + dt
        du = cols[None, :] - (rec[0] + rec[7] * times[:, None])
        dv = rows[:, None] - (rec[1] + rec[8] * times[:, None])
        alpha = rec[5] * np.exp(-0.5 * _form(rec, du, dv))
        assert alpha.max() < A_MIN


def test_culled_lists_are_the_box_lists_without_the_culled_pairs():
    g, cam = _moving_scene(seed=7)
    t0, i0 = oracle.isect_list(g, cam)
    t1, i1 = oracle.isect_list(g, _cull(cam))
    assert len(t1) < 0.9 * len(t0)
    marg = oracle.tile_margin(g, _cull(cam), t0, i0)
    keep = marg <= 0
    np.testing.assert_array_equal(t1, t0[keep])
    np.testing.assert_array_equal(i1, i0[keep])


def test_the_cull_never_changes_a_render():
    for seed in (3, 9):
        g, cam = _moving_scene(seed=seed)
        a = oracle.render(g, cam)
        b = oracle.render(g, _cull(cam))
        np.testing.assert_array_equal(a["F"], b["F"])
        np.testing.assert_array_equal(a["T"], b["T"])
        np.testing.assert_array_equal(a["count"], b["count"])


def test_the_cull_applies_to_cameras_only():
    g, sensors = scenes.tiny_frame()
    lid = sensors[1]
    t0, i0 = oracle.isect_list(g, lid)
    t1, i1 = oracle.isect_list(g, dataclasses.replace(lid, support=4))
    np.testing.assert_array_equal(t0, t1)
    np.testing.assert_array_equal(i0, i1)
