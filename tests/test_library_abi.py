"""The C-ABI library builds, loads and exports every entry point include/splat.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2411_16816_gb300 import _lib as L
from paper_2411_16816_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "splat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(splat_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_contract():
    syms = _declared_symbols()
    for name in ("splat_project", "splat_bin_sort", "splat_render_camera", "splat_render_lidar",
                 "splat_project_backward", "splat_bin_sort_backward", "splat_render_camera_backward",
                 "splat_render_lidar_backward"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    lib = L.load()
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    assert set(_declared_symbols()) <= set(L.EXPORTS) | {"splat_bin_sort_noalloc"}


def test_struct_layout_matches_header():
    # offsets computed by hand from the C declaration order and natural alignment
    assert ctypes.sizeof(L.splat_gaussians) == 64
    assert L.splat_sensor.beam_elev.offset == 128
    assert ctypes.sizeof(L.splat_sensor) == 168
    assert ctypes.sizeof(L.splat_projected) == 24 and ctypes.sizeof(L.splat_bins) == 24


def _c_sensor(s):
    c = L.splat_sensor()
    c.kind = 0 if s.kind == "camera" else 1
    c.R[:] = list(np.asarray(s.R, np.float32).reshape(9))
    if s.kind == "camera":
        c.width, c.height, c.fx, c.fy, c.cx, c.cy = s.width, s.height, s.fx, s.fy, s.cx, s.cy
        c.tile_w, c.tile_h, c.eps2d = s.tile_w, s.tile_h, s.eps2d
    else:
        c.n_beams, c.n_az, c.az_res, c.tile_w, c.tile_h = s.n_beams, s.n_az, s.az_res, s.tile_az, s.tile_el
        c.beam_elev = 0x1000   # never dereferenced by layout queries
        c.eps2d = s.eps2d
    return c


def test_frame_layout_counts_tiles_and_rays():
    lib = L.load()
    g, sensors = scenes.tiny_frame()
    arr = (L.splat_sensor * 2)(*[_c_sensor(s) for s in sensors])
    total = ctypes.c_int64()
    tiles = (ctypes.c_int64 * 2)()
    rays = (ctypes.c_int64 * 2)()
    assert lib.splat_frame_layout(2, arr, ctypes.byref(total), tiles, rays) == 0
    assert list(tiles) == [8 * 6, 8 * 2] and total.value == 64
    assert list(rays) == [128 * 96, 16 * 256]
    ws, ws2 = ctypes.c_size_t(), ctypes.c_size_t()
    # visible-pair keys and values, double-buffered: at least 16 bytes per (sensor, Gaussian)
    assert lib.splat_workspace_size(2000, 2, arr, 100000, ctypes.byref(ws)) == 0 and ws.value >= 16 * 2 * 2000
    assert lib.splat_workspace_size(4000, 2, arr, 100000, ctypes.byref(ws2)) == 0 and ws2.value > ws.value


@pytest.mark.parametrize("mutate, msg", [
    (lambda c: setattr(c, "tile_w", 7), "unsupported tile"),
    (lambda c: setattr(c, "width", 0), "bad size"),
    (lambda c: setattr(c, "kind", 5), "bad kind"),
])
def test_invalid_camera_rejected_on_host(mutate, msg):
    lib = L.load()
    c = _c_sensor(scenes.tiny_frame()[1][0])
    mutate(c)
    arr = (L.splat_sensor * 1)(c)
    total = ctypes.c_int64()
    assert lib.splat_frame_layout(1, arr, ctypes.byref(total), None, None) == L.SPLAT_ERR_INVALID_ARG
    assert msg in lib.splat_last_error().decode()


def test_invalid_lidar_rejected_on_host():
    lib = L.load()
    lid = scenes.tiny_frame()[1][1]
    c = _c_sensor(lid)
    c.tile_h = 5          # 16 beams are not a multiple of 5
    arr = (L.splat_sensor * 1)(c)
    assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_ERR_INVALID_ARG
    c = _c_sensor(lid)
    c.az_res = float(2 * math.pi / 200)   # 256 bins do not cover the circle
    arr = (L.splat_sensor * 1)(c)
    assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_ERR_INVALID_ARG
    assert "2 pi" in lib.splat_last_error().decode()


def test_too_many_sensors_rejected():
    lib = L.load()
    c = _c_sensor(scenes.tiny_frame()[1][0])
    arr = (L.splat_sensor * 17)(*([c] * 17))
    assert lib.splat_frame_layout(17, arr, None, None, None) == L.SPLAT_ERR_INVALID_ARG


def test_bin_sort_rejects_small_workspace_before_launch():
    lib = L.load()
    c = _c_sensor(scenes.tiny_frame()[1][0])
    arr = (L.splat_sensor * 1)(c)
    proj = L.splat_projected(0x1000, 0x1000, 0x1000)
    bins = L.splat_bins(0x1000, 0x1000, 0x1000)
    st = lib.splat_bin_sort(10, 1, arr, proj, 100, bins, ctypes.c_void_p(0x1000), 16, None)
    assert st == L.SPLAT_ERR_INVALID_ARG and "workspace too small" in lib.splat_last_error().decode()


def test_point_cloud_entry_points_check_arguments_on_host():
    """The free-ray entry points (App. A.2) reject a camera index, an out-of-range count
    and missing buffers before any launch."""
    lib = L.load()
    cam, lid = scenes.tiny_frame()[1]
    arr = (L.splat_sensor * 2)(_c_sensor(cam), _c_sensor(lid))
    p = ctypes.c_void_p(0x1000)
    st = lib.splat_lidar_points_to_rays(2, arr, 0, p, p, 10, p, p, None, None)
    assert st == L.SPLAT_ERR_INVALID_ARG and "not a lidar" in lib.splat_last_error().decode()
    st = lib.splat_lidar_points_to_rays(2, arr, 1, p, p, 1 << 31, p, p, None, None)
    assert st == L.SPLAT_ERR_INVALID_ARG
    st = lib.splat_lidar_points_to_rays(2, arr, 1, None, p, 10, p, p, None, None)
    assert st == L.SPLAT_ERR_INVALID_ARG and "required" in lib.splat_last_error().decode()
    bins = L.splat_ray_bins(0x1000, 0x1004, 0x1000)   # tile ranges not 8-byte aligned
    st = lib.splat_lidar_bin_rays(2, arr, 1, p, 10, bins, None)
    assert st == L.SPLAT_ERR_INVALID_ARG and "aligned" in lib.splat_last_error().decode()
    bins = L.splat_ray_bins(None, 0x1000, 0x1000)
    st = lib.splat_lidar_bin_rays(2, arr, 1, p, 10, bins, None)
    assert st == L.SPLAT_ERR_INVALID_ARG and "NULL" in lib.splat_last_error().decode()
    assert ctypes.sizeof(L.splat_ray_bins) == 24


def test_support_flags_checked_on_host():
    """Unknown extent flags, and the sweep-time flag on a camera or on a lidar with an
    explicit ray table, are refused before any launch; the camera tile cull (4) is
    accepted on cameras and on lidars, where it has no effect."""
    lib = L.load()
    cam, lid = scenes.tiny_frame()[1]
    for s, flags in ((cam, 8), (cam, 2), (lid, 8)):
        c = _c_sensor(s)
        c.support = flags
        arr = (L.splat_sensor * 1)(c)
        assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_ERR_INVALID_ARG, (s.kind, flags)
    for s, flags in ((cam, 5), (lid, 4), (lid, 6)):
        c = _c_sensor(s)
        c.support = flags
        arr = (L.splat_sensor * 1)(c)
        assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_OK, (s.kind, flags)
    c = _c_sensor(lid)
    c.support = 2
    c.rays = 0x1000
    arr = (L.splat_sensor * 1)(c)
    assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_ERR_INVALID_ARG
    c.rays = None
    c.support = 3
    arr = (L.splat_sensor * 1)(c)
    assert lib.splat_frame_layout(1, arr, None, None, None) == L.SPLAT_OK


def test_count_nonfinite_checks_arguments_on_host():
    lib = L.load()
    g = L.splat_gaussians(0x1000, 0x1000, 0x1000, 0x1000, 0x1000, None, 10, 3, 0)
    assert lib.splat_count_nonfinite(ctypes.byref(g), None, None) == L.SPLAT_ERR_INVALID_ARG
    assert "count" in lib.splat_last_error().decode()
    assert lib.splat_count_nonfinite(ctypes.byref(g), ctypes.c_void_p(0x1004), None) == L.SPLAT_ERR_INVALID_ARG
    bad = L.splat_gaussians(None, 0x1000, 0x1000, 0x1000, 0x1000, None, 10, 3, 0)
    assert lib.splat_count_nonfinite(ctypes.byref(bad), ctypes.c_void_p(0x1000), None) == L.SPLAT_ERR_INVALID_ARG


def test_checked_build_exports_the_same_symbols_and_says_so():
    plain = L.load()
    checked = L.load(checked=True)
    assert os.path.basename(L.library_path(checked=True)) == "libsplat_checked.so"
    for name in _declared_symbols():
        assert hasattr(checked, name), name
    assert plain.splat_build_flags() == 0
    assert checked.splat_build_flags() == 1

