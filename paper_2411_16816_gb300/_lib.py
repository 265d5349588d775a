"""ctypes binding of libsplat's C ABI (include/splat.h): the same entry points and
structs, argument marshalling only.  Every computation runs in the library's CUDA
kernels; if the library cannot be loaded this module raises instead of falling back.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

from . import build as _build

c_int32, c_int64, c_float, c_void_p, c_size_t = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t

SPLAT_OK = 0
SPLAT_ERR_INVALID_ARG = 1
SPLAT_ERR_CAPACITY = 2
SPLAT_ERR_CUDA = 3
SPLAT_ERR_TIMEOUT = 4
SPLAT_ERR_BOUNDS = 5
SPLAT_SENSOR_CAMERA = 0
SPLAT_SENSOR_LIDAR = 1
SPLAT_MAX_SENSORS = 16

EXPORTS = [
    "splat_frame_layout", "splat_workspace_size", "splat_project", "splat_count_nonfinite", "splat_bin_sort",
    "splat_bin_sort_backward",
    "splat_render_camera", "splat_render_camera_l1", "splat_render_lidar", "splat_render_lidar_los",
    "splat_render_lidar_head",
    "splat_render_camera_backward", "splat_render_lidar_backward", "splat_render_lidar_backward_los",
    "splat_sync_status", "splat_lidar_points_to_rays", "splat_lidar_bin_rays", "splat_lidar_bin_rays_capped",
    "splat_render_lidar_rays",
    "splat_render_lidar_rays_backward",
    "splat_project_backward", "splat_l1_loss", "splat_last_error", "splat_head_param_count", "splat_head_inputs",
    "splat_head_forward", "splat_head_train", "splat_head_adam", "splat_batch_table_bytes", "splat_batch_build",
    "splat_render_batch", "splat_stamp", "splat_build_flags",
]


class splat_gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacities", c_void_p),
                ("features", c_void_p), ("velocities", c_void_p), ("n", c_int64), ("channels", c_int32),
                ("reserved", c_int32)]


class splat_sensor(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved0", c_int32), ("R", c_float * 9), ("t", c_float * 3),
                ("lin_vel", c_float * 3), ("ang_vel", c_float * 3), ("width", c_int32), ("height", c_int32),
                ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float), ("rs_time", c_float),
                ("time_offset", c_float), ("eps2d", c_float), ("near_plane", c_float), ("n_beams", c_int32),
                ("n_az", c_int32), ("beam_elev", c_void_p), ("rays", c_void_p), ("az_res", c_float),
                ("sweep_time", c_float), ("r_min", c_float), ("tile_w", c_int32), ("tile_h", c_int32),
                ("support", c_int32)]


class splat_projected(ctypes.Structure):
    _fields_ = [("rec", c_void_p), ("rect", c_void_p), ("n_tiles", c_void_p)]


class splat_bins(ctypes.Structure):
    _fields_ = [("isect_ids", c_void_p), ("tile_ranges", c_void_p), ("n_isect", c_void_p)]


class splat_los(ctypes.Structure):
    _fields_ = [("target_range", c_void_p), ("eps", c_float), ("reserved", c_int32)]


class splat_ray_bins(ctypes.Structure):
    _fields_ = [("ray_ids", c_void_p), ("tile_ranges", c_void_p), ("chunk_base", c_void_p)]


class splat_batch_request(ctypes.Structure):
    _fields_ = [("group_sensors", ctypes.POINTER(splat_sensor)), ("group_n_sensors", c_int32),
                ("group_sensor_index", c_int32), ("proj", splat_projected), ("bins", splat_bins),
                ("features", c_void_p), ("n", c_int64), ("channels", c_int32), ("reserved", c_int32),
                ("out_feat", c_void_p), ("out_T", c_void_p), ("out_range_exp", c_void_p),
                ("out_range_med", c_void_p), ("out_alpha", c_void_p)]


_libs = {}


class SplatError(RuntimeError):
    pass


def library_path(checked: bool = False) -> str:
    return _build.lib_path(checked)


def load(build_if_missing: bool = True, checked: bool = False):
    """Load libsplat.so (building it in-tree if it is missing or stale); with checked=True
    the checked build libsplat_checked.so, whose kernels check every index against its
    buffer and report a failing check through splat_sync_status (SPLAT_ERR_BOUNDS)."""
    if checked in _libs:
        return _libs[checked]
    path = _build.lib_path(checked)
    if build_if_missing:
        path = _build.build(checked=checked)
    if not os.path.exists(path):
        raise SplatError(f"{os.path.basename(path)} not found at {path}; run paper_2411_16816_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, S = ctypes.POINTER, c_int32
    G, SE = P(splat_gaussians), P(splat_sensor)
    L.splat_frame_layout.argtypes = [c_int32, SE, P(c_int64), P(c_int64), P(c_int64)]
    L.splat_workspace_size.argtypes = [c_int64, c_int32, SE, c_int64, P(c_size_t)]
    L.splat_project.argtypes = [G, c_int32, SE, splat_projected, c_void_p]
    L.splat_count_nonfinite.argtypes = [G, c_void_p, c_void_p]
    L.splat_bin_sort.argtypes = [c_int64, c_int32, SE, splat_projected, c_int64, splat_bins, c_void_p, c_size_t,
                                 c_void_p]
    L.splat_bin_sort_backward.argtypes = []
    L.splat_render_camera.argtypes = [G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 5
    L.splat_render_camera_l1.argtypes = [G, c_int32, SE, splat_projected, splat_bins, c_void_p, c_float] + [c_void_p] * 7
    L.splat_sync_status.argtypes = [c_void_p]
    L.splat_render_lidar_los.argtypes = ([G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 6 +
                                         [splat_los, c_void_p, c_void_p, c_void_p])
    L.splat_render_lidar_backward_los.argtypes = ([G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 5 +
                                                  [splat_los] + [c_void_p] * 4)
    L.splat_render_lidar.argtypes = [G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 8
    L.splat_render_lidar_head.argtypes = [G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 10
    L.splat_lidar_points_to_rays.argtypes = [c_int32, SE, c_int32, c_void_p, c_void_p, c_int64] + [c_void_p] * 4
    L.splat_lidar_bin_rays.argtypes = [c_int32, SE, c_int32, c_void_p, c_int64, splat_ray_bins, c_void_p]
    L.splat_lidar_bin_rays_capped.argtypes = [c_int32, SE, c_int32, c_void_p, c_void_p, c_int64, c_int32,
                                              splat_ray_bins, splat_ray_bins, c_void_p]
    L.splat_render_lidar_rays.argtypes = ([G, c_int32, SE, c_int32, splat_projected, splat_bins, c_void_p, c_int64,
                                           splat_ray_bins] + [c_void_p] * 6 + [P(splat_los), c_void_p, c_void_p])
    L.splat_render_lidar_rays_backward.argtypes = ([G, c_int32, SE, c_int32, splat_projected, splat_bins, c_void_p,
                                                    c_int64, splat_ray_bins] + [c_void_p] * 5 +
                                                   [P(splat_los)] + [c_void_p] * 4)
    L.splat_render_camera_backward.argtypes = [G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 8
    L.splat_render_lidar_backward.argtypes = [G, c_int32, SE, splat_projected, splat_bins] + [c_void_p] * 8
    L.splat_project_backward.argtypes = [G, c_int32, SE, splat_projected] + [c_void_p] * 8
    L.splat_l1_loss.argtypes = [c_void_p, c_void_p, c_int64, c_float, c_void_p, c_void_p, c_void_p]
    L.splat_head_param_count.argtypes = []
    L.splat_head_inputs.argtypes = [SE, c_void_p, c_int32, c_void_p, c_void_p]
    L.splat_head_forward.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]
    L.splat_head_train.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_float,
                                   c_void_p, c_void_p, c_void_p, c_void_p]
    L.splat_head_adam.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_float, c_float, c_float,
                                  c_int64, c_void_p, c_void_p, c_void_p]
    L.splat_batch_table_bytes.argtypes = [c_int32]
    L.splat_batch_table_bytes.restype = c_size_t
    L.splat_batch_build.argtypes = [P(splat_batch_request), c_int32, c_void_p, c_size_t, P(c_int64)]
    L.splat_render_batch.argtypes = [c_void_p, c_int32, c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]
    L.splat_stamp.argtypes = [c_void_p, c_void_p]
    L.splat_build_flags.argtypes = []
    L.splat_last_error.argtypes = []
    L.splat_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("splat_last_error", "splat_batch_table_bytes", "splat_head_param_count"):
            getattr(L, name).restype = S
    L.splat_head_param_count.restype = c_int32
    _libs[checked] = L
    return L


_active_checked = [False]


@contextlib.contextmanager
def checked_build():
    """Within the block, call() and check() go to the checked build (load(checked=True))."""
    prev = _active_checked[0]
    _active_checked[0] = True
    try:
        yield load(checked=True)
    finally:
        _active_checked[0] = prev


def active():
    """The library call() uses: the checked build inside checked_build(), else libsplat.so."""
    return load(checked=_active_checked[0])


def check(status: int, what: str = "") -> None:
    if status != SPLAT_OK:
        msg = load(checked=_active_checked[0]).splat_last_error().decode()
        raise SplatError(f"{what} failed with status {status}: {msg}")


def call(name: str, *args) -> None:
    """Call a libsplat entry point and raise on a non-OK status."""
    check(getattr(load(checked=_active_checked[0]), name)(*args), name)
