"""splat_bin_sort_noalloc: the binning sort for callers that cannot allocate device memory
(hosts with a fixed device-memory budget, plug-ins inside another program's frame loop,
runtimes that forbid allocation after start-up).  It takes its scratch from an array
built into the library instead of a caller workspace; its lists must equal those of
splat_bin_sort exactly, call after call, even though every call reuses the same array.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_16816_gb300 import _lib as L
from paper_2411_16816_gb300 import scenes
from paper_2411_16816_gb300.render import Frame, _stream, gaussians_to_device
from tests.helpers import front_camera, small_lidar

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _entry():
    f = L.load().splat_bin_sort_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(L.splat_sensor), L.splat_projected,
                  ctypes.c_int64, L.splat_bins, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return f


def _frames():
    g, sensors = scenes.tiny_frame()
    yield g, sensors
    g2, _ = scenes.tiny_frame(seed=4242)
    rng = np.random.default_rng(5)
    g2 = dict(g2)
    g2["velocities"] = rng.normal(0, 2.0, size=(len(g2["opacities"]), 3)).astype(np.float32)
    cam = front_camera(rs_time=0.03, lin_vel=np.array([0.5, 0.0, 10.0]))
    lid = small_lidar(n_az=1000, sweep_time=0.1, lin_vel=np.array([10.0, 0.0, 0.0]))
    yield g2, [cam, lid]


def test_noalloc_bin_sort_equals_workspace_bin_sort_on_repeated_calls():
    entry = _entry()
    for g, sensors in _frames():
        gd = gaussians_to_device(g, DEV)
        fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
        fr.forward(gd)                      # project + splat_bin_sort with a caller workspace
        torch.cuda.synchronize()
        n_ref = int(fr.n_isect.item())
        ids_ref = fr.isect_ids[:n_ref].clone()
        ranges_ref = fr.ranges.clone()
        ids = torch.empty_like(fr.isect_ids)
        ranges = torch.empty_like(fr.ranges)
        n_out = torch.empty(1, dtype=torch.int64, device=DEV)
        bins = L.splat_bins(ids.data_ptr(), ranges.data_ptr(), n_out.data_ptr())
        for call in range(2):
            ids.fill_(-1)
            ranges.fill_(-7)
            n_out.fill_(-1)
            st = entry(fr.n, len(fr.sensors), fr.c_sensors, fr.c_proj(), fr.capacity, bins, _stream())
            assert st == L.SPLAT_OK, L.load().splat_last_error().decode()
            torch.cuda.synchronize()
            assert int(n_out.item()) == n_ref, f"call {call}"
            assert torch.equal(ids[:n_ref], ids_ref), f"call {call}: lists differ"
            assert torch.equal(ranges, ranges_ref), f"call {call}: tile ranges differ"


def test_noalloc_rejects_a_frame_beyond_its_scratch():
    entry = _entry()
    # 2M Gaussians x 7 sensors: the visible-pair buffers alone are far above 32 MiB
    g, sensors = scenes.driving_frame(n=2_000_000)
    fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV, capacity=1 << 22)
    fr.project(fr.c_gaussians(gaussians_to_device(g, DEV)))   # valid inputs even though it must refuse
    torch.cuda.synchronize()
    bins = L.splat_bins(fr.isect_ids.data_ptr(), fr.ranges.data_ptr(), fr.n_isect.data_ptr())
    st = entry(fr.n, len(fr.sensors), fr.c_sensors, fr.c_proj(), fr.capacity, bins, _stream())
    assert st == L.SPLAT_ERR_INVALID_ARG
    assert "scratch" in L.load().splat_last_error().decode()
