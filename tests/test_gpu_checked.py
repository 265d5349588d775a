"""The checked build (libsplat_checked.so, compiled with SPLAT_CHECKED).

Every kernel of that build checks the indices it reads from its inputs against their
buffers (tile ranges against the list's length, listed Gaussian and ray indices against
their counts, scatter and binning slots against theirs).  A failing check skips the access
and raises the device status word, which splat_sync_status reports as SPLAT_ERR_BOUNDS with
the first failing site.  On well-formed inputs the build must give the normal build's
results; on lists holding an out-of-range tile range or index it must report the site.
The malformed lists are only ever given to the checked build (each test asserts which
library it is calling before it does so).
"""
import contextlib
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2411_16816_gb300 import _lib as L
from paper_2411_16816_gb300 import scenes
from paper_2411_16816_gb300.render import Frame, gaussians_to_device
from tests.test_gpu_parity import _cull_cameras, _dynamic_tiny, _point_cloud, _small_driving

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _seeded_like(t, seed):
    gen = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(t.shape, generator=gen, dtype=torch.float32).to(t.device)


def _run(checked, g, sensors, pts, times):
    """Forward and backward of the grid rays and of a point cloud's free rays."""
    ctx = L.checked_build() if checked else contextlib.nullcontext()
    res = {}
    with ctx:
        lib = L.active()
        assert lib.splat_build_flags() == int(checked)
        gd = gaussians_to_device(g, DEV)
        fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
        out = fr.forward(gd)
        grads = {k: _seeded_like(out[k], i) for i, k in enumerate(("cam_feat", "lid_feat", "lid_range_exp"))}
        pg = fr.backward(gd, out, grads)
        res.update({"fwd_" + k: v.clone() for k, v in out.items() if v is not None})
        res.update({"bwd_" + k: v.clone() for k, v in pg.items() if v is not None})
        pr = fr.lidar_points_to_rays(1, torch.as_tensor(pts, device=DEV), torch.as_tensor(times, device=DEV))
        b = fr.bin_rays(1, pr["rays"])
        cg = fr.prepare(gd)
        o2 = fr.render_rays(cg, 1, pr["rays"], b)
        res.update({"rays_" + k: v.clone() for k, v in o2.items() if v is not None})
        pg2 = fr.backward_rays(gd, 1, pr["rays"], b, o2, {"feat": _seeded_like(o2["feat"], 7)})
        res.update({"raysbwd_" + k: v.clone() for k, v in pg2.items() if v is not None})
        st = lib.splat_sync_status(_stream())
    return res, st


def test_checked_build_gives_the_normal_builds_results():
    g, sensors = _dynamic_tiny()
    pts, times = _point_cloud(sensors[1], 6000, 21)
    a, sa = _run(False, g, sensors, pts, times)
    b, sb = _run(True, g, sensors, pts, times)
    assert sa == L.SPLAT_OK and sb == L.SPLAT_OK
    assert a.keys() == b.keys()
    for k in a:
        if k.startswith(("fwd_", "rays_")):
            # forward passes are deterministic: bit for bit
            assert torch.equal(a[k], b[k]), k
        else:
            # gradients are accumulated with atomics in an arbitrary order
            scale = float(a[k].abs().max()) + 1e-30
            assert float((a[k] - b[k]).abs().max()) <= 1e-5 * scale, k


def _prepared_checked():
    g, sensors = scenes.tiny_frame()
    gd = gaussians_to_device(g, DEV)
    fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
    cg = fr.prepare(gd)
    return fr, gd, cg


def test_checked_build_reports_a_tile_range_past_the_list_and_a_gaussian_index_past_the_gaussians():
    with L.checked_build():
        lib = L.active()
        assert lib.splat_build_flags() == 1   # the malformed lists below go to the checked build only
        fr, gd, cg = _prepared_checked()
        ref = fr.alloc_outputs()
        fr.rasterize(cg, ref)
        assert lib.splat_sync_status(_stream()) == L.SPLAT_OK
        n = int(fr.n_isect.item())
        ranges = fr.ranges.clone()
        lens = (ranges[:, 1] - ranges[:, 0]).cpu().numpy()
        t = int(np.argmax(lens))
        assert lens[t] > 0

        # a tile range reaching past the list's length
        fr.ranges[t, 1] = n + 1000
        out = fr.alloc_outputs()
        fr.rasterize(cg, out)
        st = lib.splat_sync_status(_stream())
        msg = lib.splat_last_error().decode()
        assert st == L.SPLAT_ERR_BOUNDS and "(site 1)" in msg, (st, msg)
        fr.ranges.copy_(ranges)

        # a listed Gaussian index past the Gaussians
        j = int(ranges[t, 0])
        saved = fr.isect_ids[j].clone()
        fr.isect_ids[j] = fr.n + 7
        out = fr.alloc_outputs()
        fr.rasterize(cg, out)
        st = lib.splat_sync_status(_stream())
        msg = lib.splat_last_error().decode()
        assert st == L.SPLAT_ERR_BOUNDS and "(site 2)" in msg, (st, msg)
        fr.isect_ids[j] = saved

        # restored lists: clean status and the first render again
        out = fr.alloc_outputs()
        fr.rasterize(cg, out)
        assert lib.splat_sync_status(_stream()) == L.SPLAT_OK
        for k in ref:
            if ref[k] is not None:
                assert torch.equal(out[k], ref[k]), k


def test_checked_build_reports_a_ray_index_past_the_rays():
    g, sensors = _dynamic_tiny()
    pts, times = _point_cloud(sensors[1], 3000, 5)
    with L.checked_build():
        lib = L.active()
        assert lib.splat_build_flags() == 1
        gd = gaussians_to_device(g, DEV)
        fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
        pr = fr.lidar_points_to_rays(1, torch.as_tensor(pts, device=DEV), torch.as_tensor(times, device=DEV))
        b = fr.bin_rays(1, pr["rays"])
        cg = fr.prepare(gd)
        fr.render_rays(cg, 1, pr["rays"], b)
        assert lib.splat_sync_status(_stream()) == L.SPLAT_OK
        b["ray_ids"][0] = pr["rays"].shape[0] + 3
        fr.render_rays(cg, 1, pr["rays"], b)
        st = lib.splat_sync_status(_stream())
        msg = lib.splat_last_error().decode()
        assert st == L.SPLAT_ERR_BOUNDS and "(site 4)" in msg, (st, msg)


def _driving16(cull):
    """Two 320 x 180 rolling-shutter cameras and the lidar, 16 channels: the camera backward
    of the 16-channel bucket on 256-ray tiles (tensor cores); with the camera tile cull its
    unpacked staging, without it the packing one."""
    g, sensors = _small_driving(n=20000, w=320, h=180, box=30)
    return g, (_cull_cameras(sensors) if cull else sensors)


def _run16(checked, g, sensors):
    ctx = L.checked_build() if checked else contextlib.nullcontext()
    with ctx:
        lib = L.active()
        assert lib.splat_build_flags() == int(checked)
        gd = gaussians_to_device(g, DEV)
        fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
        out = fr.forward(gd)
        grads = {k: _seeded_like(out[k], i) for i, k in enumerate(("cam_feat", "lid_feat", "lid_range_exp"))}
        pg = fr.backward(gd, out, grads)
        res = {"fwd_" + k: v.clone() for k, v in out.items() if v is not None}
        res.update({"bwd_" + k: v.clone() for k, v in pg.items() if v is not None})
        st = lib.splat_sync_status(_stream())
    return res, st


@pytest.mark.parametrize("cull", [False, True])
def test_checked_build_gives_the_normal_builds_results_with_16_channels(cull):
    g, sensors = _driving16(cull)
    a, sa = _run16(False, g, sensors)
    b, sb = _run16(True, g, sensors)
    assert sa == L.SPLAT_OK and sb == L.SPLAT_OK
    assert a.keys() == b.keys()
    for k in a:
        if k.startswith("fwd_"):
            assert torch.equal(a[k], b[k]), k
        else:
            # atomic sums in an arbitrary order over many more (tile, Gaussian) terms than the
            # tiny frame's: the quaternion gradients differ by up to about 1.3e-5 of their
            # largest element between two builds
            scale = float(a[k].abs().max()) + 1e-30
            assert float((a[k] - b[k]).abs().max()) <= 1e-4 * scale, k


@pytest.mark.parametrize("cull", [False, True])
def test_checked_build_reports_a_gaussian_index_past_the_gaussians_in_the_16_channel_backward(cull):
    with L.checked_build():
        lib = L.active()
        assert lib.splat_build_flags() == 1   # the malformed list below goes to the checked build only
        g, sensors = _driving16(cull)
        gd = gaussians_to_device(g, DEV)
        fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV)
        out = fr.forward(gd)
        grads = {k: _seeded_like(out[k], i) for i, k in enumerate(("cam_feat", "lid_feat", "lid_range_exp"))}
        assert lib.splat_sync_status(_stream()) == L.SPLAT_OK
        # the longest list of the first camera (its tiles come first)
        ranges = fr.ranges.clone()
        n_cam0 = oracle.n_tiles_of(sensors[0])
        lens = (ranges[:n_cam0, 1] - ranges[:n_cam0, 0]).cpu().numpy()
        t = int(np.argmax(lens))
        assert lens[t] > 0
        j = int(ranges[t, 0])
        saved = fr.isect_ids[j].clone()
        fr.isect_ids[j] = fr.n + 7
        fr.backward(gd, out, grads)
        st = lib.splat_sync_status(_stream())
        msg = lib.splat_last_error().decode()
        assert st == L.SPLAT_ERR_BOUNDS and "(site 2)" in msg, (st, msg)
        fr.isect_ids[j] = saved
        fr.backward(gd, out, grads)
        assert lib.splat_sync_status(_stream()) == L.SPLAT_OK
