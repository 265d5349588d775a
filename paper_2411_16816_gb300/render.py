"""Torch-facing wrapper of libsplat: device buffers, the per-frame call sequence and
the autograd function.

PyTorch only provides device memory and the stream here; every step of the
projection, binning, rasterization and backward runs in libsplat's CUDA kernels
(called through :mod:`._lib`).  There is no CPU path.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib as L

_PARAMS = ("means", "scales", "quats", "opacities", "features", "velocities")


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _f32(a, device):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)


def gaussians_to_device(g: dict, device="cuda") -> dict:
    """Copy a dict of numpy arrays (see scenes.py) to contiguous FP32 device tensors."""
    out = {}
    for k in _PARAMS:
        v = g.get(k)
        out[k] = None if v is None else _f32(v, device)
    return out


class Frame:
    """A fixed set of sensors rendered together (one projection, one sort, one raster
    launch per sensor kind).  Holds the library's per-frame device buffers for a
    scene of `n` Gaussians with `channels` features.

    `capacity` is the intersection buffer size; `forward(..., check=True)` grows it
    and re-runs the binning when the frame needs more."""

    def __init__(self, sensors, n: int, channels: int, device="cuda", capacity: int | None = None):
        if not 1 <= len(sensors) <= L.SPLAT_MAX_SENSORS:
            raise ValueError(f"a frame holds 1..{L.SPLAT_MAX_SENSORS} sensors")
        self.lib = L.active()
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.sensors = list(sensors)
        self.n, self.channels = int(n), int(channels)
        S = len(self.sensors)
        self._keep = []
        self.c_sensors = (L.splat_sensor * S)()
        for k, s in enumerate(self.sensors):
            self._fill_sensor(self.c_sensors[k], s)
        total = ctypes.c_int64()
        tiles = (ctypes.c_int64 * S)()
        rays = (ctypes.c_int64 * S)()
        L.call("splat_frame_layout", S, self.c_sensors, ctypes.byref(total), tiles, rays)
        self.total_tiles = total.value
        self.tiles = list(tiles)
        self.rays = list(rays)
        self.cam_idx = [k for k, s in enumerate(self.sensors) if s.kind == "camera"]
        self.lid_idx = [k for k, s in enumerate(self.sensors) if s.kind == "lidar"]
        self.cam_rays = sum(self.rays[k] for k in self.cam_idx)
        self.lid_rays = sum(self.rays[k] for k in self.lid_idx)
        dev = self.device
        self.rec = torch.empty((S, 3, max(self.n, 1), 4), dtype=torch.float32, device=dev)
        self.rect = torch.empty((S, max(self.n, 1), 4), dtype=torch.int16, device=dev)
        self.n_tiles = torch.empty((S, max(self.n, 1)), dtype=torch.int32, device=dev)
        self.ranges = torch.empty((max(self.total_tiles, 1), 2), dtype=torch.int32, device=dev)
        self.n_isect = torch.zeros(1, dtype=torch.int64, device=dev)
        self.capacity = 0
        self._alloc_capacity(capacity if capacity is not None else max(1 << 16, 8 * self.n))
        self.grad_proj = None
        self.los = None           # line-of-sight term: (return range per lidar ray, eps) or None
        self.version = 0
        # the lidar raster launches (a few hundred blocks) run beside the camera launches on
        # a second stream, filling the SMs the camera grid leaves idle
        self.overlap_kinds = True
        self._side = None

    # -- set-up ------------------------------------------------------------------------
    def _fill_sensor(self, c, s):
        c.R[:] = [float(x) for x in np.asarray(s.R, dtype=np.float32).reshape(9)]
        c.t[:] = [float(x) for x in np.asarray(s.t, dtype=np.float32)]
        c.lin_vel[:] = [float(x) for x in np.asarray(s.lin_vel, dtype=np.float32)]
        c.ang_vel[:] = [float(x) for x in np.asarray(s.ang_vel, dtype=np.float32)]
        c.tile_w, c.tile_h = s.tile_w if s.kind == "camera" else s.tile_az, s.tile_h if s.kind == "camera" else s.tile_el
        c.eps2d = s.eps2d
        c.support = int(getattr(s, "support", 0))
        if s.kind == "camera":
            c.kind = L.SPLAT_SENSOR_CAMERA
            c.width, c.height = s.width, s.height
            c.fx, c.fy, c.cx, c.cy = s.fx, s.fy, s.cx, s.cy
            c.rs_time, c.time_offset, c.near_plane = s.rs_time, s.time_offset, s.near
        else:
            c.kind = L.SPLAT_SENSOR_LIDAR
            c.n_beams, c.n_az = s.n_beams, s.n_az
            elev = _f32(s.beam_elev, self.device)
            self._keep.append(elev)
            c.beam_elev = elev.data_ptr()
            if s.rays is not None:
                rays = _f32(np.asarray(s.rays).reshape(s.n_beams, s.n_az, 3), self.device)
                self._keep.append(rays)
                c.rays = rays.data_ptr()
            c.az_res, c.sweep_time, c.r_min = s.az_res, s.sweep_time, s.r_min

    def _alloc_capacity(self, capacity: int):
        capacity = int(max(capacity, 1))
        self.capacity = capacity
        self.isect_ids = torch.empty(capacity, dtype=torch.int32, device=self.device)
        ws = ctypes.c_size_t()
        L.call("splat_workspace_size", self.n, len(self.sensors), self.c_sensors, capacity, ctypes.byref(ws))
        self.workspace = torch.empty(max(ws.value, 256), dtype=torch.uint8, device=self.device)

    def c_gaussians(self, g: dict) -> L.splat_gaussians:
        for k in ("means", "scales", "quats", "opacities", "features"):
            t = g[k]
            if t.dtype != torch.float32 or not t.is_contiguous() or t.device != self.device:
                raise ValueError(f"{k} must be a contiguous float32 tensor on {self.device}")
        if g["means"].shape[0] != self.n or g["features"].shape[1] != self.channels:
            raise ValueError("scene size does not match the frame")
        vel = g.get("velocities")
        return L.splat_gaussians(g["means"].data_ptr(), g["scales"].data_ptr(), g["quats"].data_ptr(),
                                 g["opacities"].data_ptr(), g["features"].data_ptr(),
                                 vel.data_ptr() if vel is not None else None, self.n, self.channels, 0)

    def c_proj(self):
        return L.splat_projected(self.rec.data_ptr(), self.rect.data_ptr(), self.n_tiles.data_ptr())

    def c_bins(self):
        return L.splat_bins(self.isect_ids.data_ptr(), self.ranges.data_ptr(), self.n_isect.data_ptr())

    # -- forward ------------------------------------------------------------------------
    def project(self, cg, stream=None):
        L.call("splat_project", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(), _stream(stream))

    def count_nonfinite(self, g: dict, count: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Device int64 count of the Gaussians with a NaN or infinite mean, scale,
        quaternion, opacity or velocity (accumulated into `count` if given).  The
        projection culls exactly those (and zero quaternions) from every sensor."""
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        L.call("splat_count_nonfinite", ctypes.byref(self.c_gaussians(g)), _vp(count), _stream(stream))
        return count

    def bin_sort(self, stream=None):
        L.call("splat_bin_sort", self.n, len(self.sensors), self.c_sensors, self.c_proj(), self.capacity,
               self.c_bins(), _vp(self.workspace), self.workspace.numel(), _stream(stream))

    def ensure_capacity(self, stream=None) -> bool:
        """Reads the intersection count (one sync); grows and re-bins while it overflows
        (the first report may be the sort's row items rather than the intersections).
        Returns True if the lists had to be rebuilt."""
        grown = False
        need = int(self.n_isect.item())
        while need > self.capacity:
            self._alloc_capacity(int(need * 1.25) + 1024)
            self.bin_sort(stream)
            grown = True
            need = int(self.n_isect.item())
        return grown

    def alloc_outputs(self, keep_state: bool = True) -> dict:
        dev, C = self.device, self.channels
        out = {}
        if self.cam_idx:
            out["cam_feat"] = torch.empty((self.cam_rays, C), dtype=torch.float32, device=dev)
            out["cam_T"] = torch.empty(self.cam_rays, dtype=torch.float32, device=dev)
            out["cam_last"] = torch.empty(self.cam_rays, dtype=torch.int32, device=dev) if keep_state else None
        if self.lid_idx:
            R = self.lid_rays
            out["lid_feat"] = torch.empty((R, C), dtype=torch.float32, device=dev)
            out["lid_range_exp"] = torch.empty(R, dtype=torch.float32, device=dev)
            out["lid_range_med"] = torch.empty(R, dtype=torch.float32, device=dev)
            out["lid_alpha"] = torch.empty(R, dtype=torch.float32, device=dev)
            out["lid_T"] = torch.empty(R, dtype=torch.float32, device=dev) if keep_state else None
            out["lid_last"] = torch.empty(R, dtype=torch.int32, device=dev) if keep_state else None
        return out

    def _fork(self, stream):
        """(main stream handle, lidar stream handle, join) -- the lidar launches go to a
        second stream ordered after everything before on `stream`; join() makes `stream`
        wait for them."""
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        if not (self.overlap_kinds and self.cam_idx and self.lid_idx):
            h = ctypes.c_void_p(main.cuda_stream)
            return h, h, lambda: None
        if self._side is None:
            self._side = torch.cuda.Stream(device=self.device)
        side = self._side
        side.wait_stream(main)

        def join():
            main.wait_stream(side)
        return ctypes.c_void_p(main.cuda_stream), ctypes.c_void_p(side.cuda_stream), join

    def rasterize(self, cg, out: dict, stream=None, evaluated: torch.Tensor | None = None, cam_l1=None):
        """Camera and lidar raster launches.  `evaluated` (optional int64[2] device tensor)
        accumulates the examined (ray, Gaussian) pairs of the camera and lidar launch.
        `cam_l1` = (target, scale, grad, loss) fuses the camera L1 term into the camera
        launch: loss += scale * sum |F - target| and grad = scale * sign(F - target)."""
        if self.lid_idx and self.los is not None and out.get("lid_los") is None:
            out["lid_los"] = torch.empty(self.lid_rays, dtype=torch.float32, device=self.device)
        st, st_l, join = self._fork(stream)
        ev_c = ev_l = None
        if evaluated is not None:
            ev_c, ev_l = evaluated[0:1], evaluated[1:2]
        if self.lid_idx and self.los is not None:
            L.call("splat_render_lidar_los", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
                   self.c_bins(), _vp(out["lid_feat"]), _vp(out["lid_range_exp"]), _vp(out["lid_range_med"]),
                   _vp(out["lid_alpha"]), _vp(out.get("lid_T")), _vp(out.get("lid_last")), self._c_los(),
                   _vp(out["lid_los"]), _vp(ev_l), st_l)
        elif self.lid_idx:
            L.call("splat_render_lidar", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
                   self.c_bins(), _vp(out["lid_feat"]), _vp(out["lid_range_exp"]), _vp(out["lid_range_med"]),
                   _vp(out["lid_alpha"]), _vp(out.get("lid_T")), _vp(out.get("lid_last")), _vp(ev_l), st_l)
        if self.cam_idx and cam_l1 is not None:
            target, scale, grad, loss = cam_l1
            L.call("splat_render_camera_l1", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
                   self.c_bins(), _vp(target), float(scale), _vp(out["cam_feat"]), _vp(out["cam_T"]),
                   _vp(out.get("cam_last")), _vp(grad), _vp(loss), _vp(ev_c), st)
        elif self.cam_idx:
            L.call("splat_render_camera", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
                   self.c_bins(), _vp(out["cam_feat"]), _vp(out["cam_T"]), _vp(out.get("cam_last")), _vp(ev_c), st)
        join()

    def set_line_of_sight(self, target_range: torch.Tensor | None, eps: float = 0.8):
        """Enable (or with None disable) the line-of-sight term of App. B: the lidar
        forward then also writes out["lid_los"] (summed alpha of the Gaussians blended
        before target_range - eps, one return range per lidar ray, <= 0: none) and the
        backward takes its upstream gradient as grads["lid_los"]."""
        if target_range is None:
            self.los = None
            return
        if target_range.shape != (self.lid_rays,) or target_range.dtype != torch.float32:
            raise ValueError("target_range must be float32 with one entry per lidar ray")
        self.los = (target_range.contiguous(), float(eps))

    def _c_los(self):
        return L.splat_los(self.los[0].data_ptr(), self.los[1], 0)

    def prepare(self, g: dict, check: bool = True, stream=None):
        """Project and bin (the per-frame lists every raster launch reads)."""
        cg = self.c_gaussians(g)
        self.project(cg, stream)
        self.bin_sort(stream)
        if check:
            self.ensure_capacity(stream)
        return cg

    def forward(self, g: dict, keep_state: bool = True, check: bool = True, out: dict | None = None,
                stream=None, cam_l1=None) -> dict:
        """Project, bin and rasterize every sensor.  With keep_state the per-ray final
        transmittance and last index are kept for the backward pass; without it the
        backward recomputes them per tile.  cam_l1 as for rasterize()."""
        cg = self.prepare(g, check, stream)
        out = self.alloc_outputs(keep_state) if out is None else out
        self.rasterize(cg, out, stream, cam_l1=cam_l1)
        self.version += 1
        return out

    def split(self, flat: torch.Tensor, kind: str):
        """Per-sensor views of a concatenated output (cameras H x W [x C], lidars B x A [x C])."""
        idx = self.cam_idx if kind == "camera" else self.lid_idx
        views, off = [], 0
        for k in idx:
            s = self.sensors[k]
            shape = (s.height, s.width) if kind == "camera" else (s.n_beams, s.n_az)
            n = self.rays[k]
            v = flat[off:off + n]
            views.append(v.reshape(*shape, *flat.shape[1:]))
            off += n
        return views

    # -- backward -----------------------------------------------------------------------
    def backward(self, g: dict, out: dict, grads: dict, param_grads: dict | None = None, stream=None,
                 sensor_grads: torch.Tensor | None = None) -> dict:
        """Gradients with respect to the Gaussian parameters (activated scales and
        opacities, unnormalised quaternions) for upstream gradients
        grads = {cam_feat, cam_T, lid_feat, lid_range_exp, lid_alpha, lid_los} (any may be
        absent).  sensor_grads (float32 [sensors][16], device, accumulated) receives the
        gradients with respect to each sensor's linear velocity (0..2), angular velocity
        (3..5), for cameras time offset (6), translation (8..10) and rotation (11..13,
        R perturbed as (I + [theta]x) R)."""
        if sensor_grads is not None and (sensor_grads.shape != (len(self.sensors), 16) or
                                         sensor_grads.dtype != torch.float32 or not sensor_grads.is_contiguous()):
            raise ValueError("sensor_grads must be a contiguous float32 [sensors][16] tensor")
        cg = self.c_gaussians(g)
        st = _stream(stream)
        dev = self.device
        if self.grad_proj is None:
            self.grad_proj = torch.zeros_like(self.rec)
        else:
            self.grad_proj.zero_()
        if param_grads is None:
            param_grads = {k: torch.zeros_like(g[k]) for k in _PARAMS if g.get(k) is not None}
        else:
            for v in param_grads.values():
                v.zero_()
        # upstream buffers on the calling stream first; then the lidar backward beside the
        # camera backward (disjoint sensor slices of grad_proj; the feature gradients are
        # atomic sums), joined before the projection backward
        dFc = dFl = dlos = None
        if self.cam_idx:
            dFc = grads.get("cam_feat")
            dFc = torch.zeros((self.cam_rays, self.channels), dtype=torch.float32, device=dev) if dFc is None \
                else dFc.contiguous()
        if self.lid_idx:
            dFl = grads.get("lid_feat")
            dFl = torch.zeros((self.lid_rays, self.channels), dtype=torch.float32, device=dev) if dFl is None \
                else dFl.contiguous()
            dlos = grads.get("lid_los")
            if dlos is not None:
                if self.los is None:
                    raise ValueError("grads['lid_los'] needs set_line_of_sight() before the forward")
                dlos = dlos.contiguous()
        st, st_l, join = self._fork(stream)
        if self.lid_idx:
            keep = out.get("lid_last") is not None
            if dlos is not None:
                L.call("splat_render_lidar_backward_los", ctypes.byref(cg), len(self.sensors), self.c_sensors,
                       self.c_proj(), self.c_bins(), _vp(out.get("lid_T") if keep else None),
                       _vp(out.get("lid_last") if keep else None), _vp(dFl),
                       _vp(grads.get("lid_range_exp")), _vp(grads.get("lid_alpha")), self._c_los(),
                       _vp(dlos), _vp(self.grad_proj), _vp(param_grads["features"]), st_l)
            else:
                L.call("splat_render_lidar_backward", ctypes.byref(cg), len(self.sensors), self.c_sensors,
                       self.c_proj(), self.c_bins(), _vp(out.get("lid_T") if keep else None),
                       _vp(out.get("lid_last") if keep else None), _vp(dFl),
                       _vp(grads.get("lid_range_exp")), _vp(grads.get("lid_alpha")), _vp(self.grad_proj),
                       _vp(param_grads["features"]), st_l)
        if self.cam_idx:
            L.call("splat_render_camera_backward", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
                   self.c_bins(), _vp(out.get("cam_T") if out.get("cam_last") is not None else None),
                   _vp(out.get("cam_last")), _vp(dFc), _vp(grads.get("cam_T")), _vp(self.grad_proj),
                   _vp(param_grads["features"]), _vp(sensor_grads), st)
        join()
        L.call("splat_project_backward", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
               _vp(self.grad_proj), _vp(param_grads["means"]), _vp(param_grads["scales"]),
               _vp(param_grads["quats"]), _vp(param_grads["opacities"]), _vp(param_grads.get("velocities")),
               _vp(sensor_grads), st)
        return param_grads

    # -- lidar point clouds as rays (App. A.2) ------------------------------------------
    def _check_lidar(self, lidar: int):
        if not 0 <= lidar < len(self.sensors) or self.sensors[lidar].kind != "lidar":
            raise ValueError(f"sensor {lidar} is not a lidar of the frame")

    def lidar_points_to_rays(self, lidar: int, points: torch.Tensor, times: torch.Tensor, stream=None) -> dict:
        """Points (n, 3; sensor frame at the sweep's reference time) and capture times (n,)
        -> {"rays": (n, 3) phi, omega, t; "ranges": (n,); "tiles": (n,) int32, -1 outside
        the beam fan}."""
        self._check_lidar(lidar)
        points = points.contiguous()
        times = times.contiguous()
        n = points.shape[0]
        if points.shape != (n, 3) or times.shape != (n,):
            raise ValueError("points must be (n, 3) and times (n,)")
        dev = self.device
        out = {"rays": torch.empty((n, 3), dtype=torch.float32, device=dev),
               "ranges": torch.empty(n, dtype=torch.float32, device=dev),
               "tiles": torch.empty(n, dtype=torch.int32, device=dev)}
        L.call("splat_lidar_points_to_rays", len(self.sensors), self.c_sensors, lidar, _vp(points), _vp(times), n,
               _vp(out["rays"]), _vp(out["ranges"]), _vp(out["tiles"]), _stream(stream))
        return out

    def _ray_bins(self, lidar: int, n: int) -> dict:
        dev, tiles = self.device, self.tiles[lidar]
        return {"ray_ids": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                "tile_ranges": torch.empty((tiles, 2), dtype=torch.int32, device=dev),
                "chunk_base": torch.empty(tiles + 1, dtype=torch.int32, device=dev), "n": n}

    def bin_rays(self, lidar: int, rays: torch.Tensor, cap: int | None = None,
                 priority: torch.Tensor | None = None, stream=None) -> dict:
        """Group free rays (n, 3) of a lidar by tile: {"ray_ids", "tile_ranges", "chunk_base"}.
        With cap (training), each tile keeps the cap rays of smallest (priority, index);
        priority (n,) int32/uint32 device values, drawn fresh per iteration."""
        self._check_lidar(lidar)
        rays = rays.contiguous()
        n = rays.shape[0]
        b = self._ray_bins(lidar, n)
        if cap is None:
            L.call("splat_lidar_bin_rays", len(self.sensors), self.c_sensors, lidar, _vp(rays), n,
                   self._c_ray_bins(b), _stream(stream))
            return b
        int_types = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
        if priority is None or priority.shape != (n,) or priority.dtype not in int_types:
            raise ValueError("a capped grouping needs one 32-bit integer priority per ray (read as unsigned)")
        priority = priority.contiguous()
        scratch = self._ray_bins(lidar, n)
        L.call("splat_lidar_bin_rays_capped", len(self.sensors), self.c_sensors, lidar, _vp(rays), _vp(priority), n,
               int(cap), self._c_ray_bins(scratch), self._c_ray_bins(b), _stream(stream))
        b["scratch"] = scratch
        return b

    @staticmethod
    def _c_ray_bins(b: dict):
        return L.splat_ray_bins(b["ray_ids"].data_ptr(), b["tile_ranges"].data_ptr(), b["chunk_base"].data_ptr())

    def render_rays(self, cg, lidar: int, rays: torch.Tensor, ray_bins: dict, keep_state: bool = True,
                    los: tuple | None = None, stream=None, out: dict | None = None) -> dict:
        """Render binned free rays of a lidar against this frame's lists (prepare() first).
        Outputs are indexed by ray; rays outside the beam fan (or dropped by a cap) keep
        their initial values (0, T = 1) -- or, with a reused `out`, the previous ones.
        los = (target_range per ray, eps) adds out["los"]."""
        self._check_lidar(lidar)
        rays = rays.contiguous()
        n, dev, C = rays.shape[0], self.device, self.channels
        if out is None:
            out = {"feat": torch.zeros((n, C), dtype=torch.float32, device=dev),
                   "range_exp": torch.zeros(n, dtype=torch.float32, device=dev),
                   "range_med": torch.zeros(n, dtype=torch.float32, device=dev),
                   "alpha": torch.zeros(n, dtype=torch.float32, device=dev),
                   "T": torch.ones(n, dtype=torch.float32, device=dev) if keep_state else None,
                   "last": torch.zeros(n, dtype=torch.int32, device=dev) if keep_state else None}
        c_los = None
        if los is not None:
            if out.get("los") is None:
                out["los"] = torch.zeros(n, dtype=torch.float32, device=dev)
            c_los = ctypes.byref(L.splat_los(los[0].data_ptr(), float(los[1]), 0))
        L.call("splat_render_lidar_rays", ctypes.byref(cg), len(self.sensors), self.c_sensors, lidar, self.c_proj(),
               self.c_bins(), _vp(rays), n, self._c_ray_bins(ray_bins), _vp(out["feat"]),
               _vp(out["range_exp"]), _vp(out["range_med"]), _vp(out["alpha"]), _vp(out["T"]), _vp(out["last"]),
               c_los, _vp(out.get("los")), _stream(stream))
        return out

    def backward_rays(self, g: dict, lidar: int, rays: torch.Tensor, ray_bins: dict, out: dict, grads: dict,
                      los: tuple | None = None, param_grads: dict | None = None, sensor_grads=None,
                      stream=None) -> dict:
        """Gradients of the free-ray render for grads = {feat, range_exp, alpha, los} (by
        ray; any may be absent), through the projection to the Gaussian parameters."""
        self._check_lidar(lidar)
        cg = self.c_gaussians(g)
        st = _stream(stream)
        rays = rays.contiguous()
        n = rays.shape[0]
        dlos = grads.get("los")
        dlos = dlos.contiguous() if dlos is not None else None
        if self.grad_proj is None:
            self.grad_proj = torch.zeros_like(self.rec)
        else:
            self.grad_proj.zero_()
        if param_grads is None:
            param_grads = {k: torch.zeros_like(g[k]) for k in _PARAMS if g.get(k) is not None}
        else:
            for v in param_grads.values():
                v.zero_()
        dF = grads.get("feat")
        dF = torch.zeros((n, self.channels), dtype=torch.float32, device=self.device) if dF is None else dF.contiguous()
        c_los = None
        if dlos is not None:
            if los is None:
                raise ValueError("grads['los'] needs the los of the forward")
            c_los = ctypes.byref(L.splat_los(los[0].data_ptr(), float(los[1]), 0))
        keep = out.get("last") is not None
        L.call("splat_render_lidar_rays_backward", ctypes.byref(cg), len(self.sensors), self.c_sensors, lidar,
               self.c_proj(), self.c_bins(), _vp(rays), n, self._c_ray_bins(ray_bins),
               _vp(out["T"] if keep else None), _vp(out["last"] if keep else None), _vp(dF),
               _vp(grads.get("range_exp")), _vp(grads.get("alpha")), c_los, _vp(dlos), _vp(self.grad_proj),
               _vp(param_grads["features"]), st)
        L.call("splat_project_backward", ctypes.byref(cg), len(self.sensors), self.c_sensors, self.c_proj(),
               _vp(self.grad_proj), _vp(param_grads["means"]), _vp(param_grads["scales"]),
               _vp(param_grads["quats"]), _vp(param_grads["opacities"]), _vp(param_grads.get("velocities")),
               _vp(sensor_grads), st)
        return param_grads

    # -- inspection ---------------------------------------------------------------------
    def intersections(self):
        """(global tile, Gaussian index) of every intersection, sorted (host arrays)."""
        n = int(self.n_isect.item())
        if n > self.capacity:
            raise RuntimeError("intersection capacity exceeded")
        ranges = self.ranges.cpu().numpy().astype(np.int64)
        ids = self.isect_ids[:n].cpu().numpy().astype(np.int64)
        full = np.nonzero(ranges[:, 1] > ranges[:, 0])[0]
        tiles = np.repeat(full, ranges[full, 1] - ranges[full, 0])
        # the non-empty ranges tile [0, n) in tile order
        if len(tiles) != n or (len(full) and (ranges[full[0], 0] != 0 or
                                              np.any(ranges[full[1:], 0] != ranges[full[:-1], 1]))):
            raise RuntimeError("tile ranges do not partition the intersection list")
        return tiles, ids


def l1_loss(pred: torch.Tensor, target: torch.Tensor, scale: float, grad: torch.Tensor | None,
            loss: torch.Tensor | None, stream=None):
    """Accumulates scale * sum|pred - target| into loss (1-element device tensor) and
    writes grad = scale * sign(pred - target) (both through libsplat)."""
    L.call("splat_l1_loss", _vp(pred), _vp(target), pred.numel(), float(scale), _vp(grad), _vp(loss),
           _stream(stream))


class RenderFrame(torch.autograd.Function):
    """Differentiable render of a Frame: inputs are the activated Gaussian parameters,
    outputs (camera features, camera T, lidar features, expected range, median range,
    lidar alpha).  With recompute=True the forward keeps no per-ray state and the
    backward recomputes it tile by tile."""

    @staticmethod
    def forward(ctx, frame: Frame, recompute: bool, means, scales, quats, opacities, features, velocities):
        g = {"means": means.detach().contiguous(), "scales": scales.detach().contiguous(),
             "quats": quats.detach().contiguous(), "opacities": opacities.detach().contiguous(),
             "features": features.detach().contiguous(),
             "velocities": velocities.detach().contiguous() if velocities is not None else None}
        out = frame.forward(g, keep_state=not recompute)
        ctx.frame, ctx.g, ctx.out, ctx.version = frame, g, out, frame.version
        ctx.has_vel = velocities is not None
        empty = torch.zeros(0, device=frame.device)
        res = (out.get("cam_feat", empty), out.get("cam_T", empty), out.get("lid_feat", empty),
               out.get("lid_range_exp", empty), out.get("lid_range_med", empty), out.get("lid_alpha", empty))
        ctx.mark_non_differentiable(res[4])
        return res

    @staticmethod
    def backward(ctx, d_cf, d_cT, d_lf, d_lr, d_lm, d_la):
        frame = ctx.frame
        if frame.version != ctx.version:
            raise RuntimeError("the Frame rendered again before this backward; use one Frame per pending graph")
        grads = {}
        if frame.cam_idx:
            grads["cam_feat"] = d_cf.contiguous() if d_cf is not None else None
            grads["cam_T"] = d_cT.contiguous() if d_cT is not None else None
        if frame.lid_idx:
            grads["lid_feat"] = d_lf.contiguous() if d_lf is not None else None
            grads["lid_range_exp"] = d_lr.contiguous() if d_lr is not None else None
            grads["lid_alpha"] = d_la.contiguous() if d_la is not None else None
        pg = frame.backward(ctx.g, ctx.out, grads)
        return (None, None, pg["means"], pg["scales"], pg["quats"], pg["opacities"], pg["features"],
                pg.get("velocities") if ctx.has_vel else None)


def render(frame: Frame, means, scales, quats, opacities, features, velocities=None, recompute=False):
    """Differentiable frame render (activated parameters).  Returns a dict of outputs."""
    cf, cT, lf, lr, lm, la = RenderFrame.apply(frame, recompute, means, scales, quats, opacities, features,
                                               velocities)
    out = {}
    if frame.cam_idx:
        out.update(cam_feat=cf, cam_T=cT)
    if frame.lid_idx:
        out.update(lid_feat=lf, lid_range_exp=lr, lid_range_med=lm, lid_alpha=la)
    return out


def render_raw(frame: Frame, means, log_scales, quats, opacity_logits, features, velocities=None, recompute=False):
    """Differentiable render from unconstrained parameters (exp scales, sigmoid opacity)."""
    return render(frame, means, torch.exp(log_scales), quats, torch.sigmoid(opacity_logits), features, velocities,
                  recompute)
