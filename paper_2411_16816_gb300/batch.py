"""Batched serving: many cameras and lidar sweeps over several scenes rendered by one
persistent launch (splat_render_batch), captured in a CUDA graph, with tile shapes
chosen by a small autotuner.

Per scene, requests are grouped into frames of at most 16 sensors that are projected
and binned with the per-frame entry points; the request table that the persistent
launch reads is built by the library on the host and copied to the device once.
"""
from __future__ import annotations

import copy
import ctypes
import itertools
import time

import numpy as np
import torch

from . import _lib as L
from .render import Frame, _stream, _vp

CAMERA_SHAPES = [(16, 16), (32, 8), (8, 32), (64, 4)]
LIDAR_SHAPES = [(32, 8), (16, 16), (64, 4)]


MAX_GROUP_TILES = 65535


def _rays(s):
    return s.n_rays


def _tiles(s):
    if s.kind == "camera":
        return (-(-s.width // s.tile_w)) * (-(-s.height // s.tile_h))
    return (-(-s.n_az // s.tile_az)) * (s.n_beams // s.tile_el)


class BatchRenderer:
    """Device state of one serving batch.  scenes: list of device Gaussian dicts (same
    channel count); requests: list of (scene index, sensor)."""

    def __init__(self, scenes, requests, cam_tile=(16, 16), lid_tile=(32, 8), device="cuda", headroom=1.25):
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.scenes = scenes
        self.C = scenes[0]["features"].shape[1]
        reqs = []
        for q, (sc, s) in enumerate(requests):
            s = copy.copy(s)
            if s.kind == "camera":
                s.tile_w, s.tile_h = cam_tile
            else:
                s.tile_az, s.tile_el = lid_tile
            reqs.append((q, sc, s))
        # largest requests first: they start early and the small ones fill the tail
        reqs.sort(key=lambda r: -_rays(r[2]))
        self.order = [r[0] for r in reqs]
        self.groups = []          # (frame, scene index, [(request position, sensor index)])
        for sc in range(len(scenes)):
            mine = [(pos, r) for pos, r in enumerate(reqs) if r[1] == sc]
            # a group holds at most 16 sensors and 65,535 tiles: its tile ids then fit 16 bits
            # and its tile sort takes two 8-bit passes
            chunks, cur, cur_tiles = [], [], 0
            for item in mine:
                t = _tiles(item[1][2])
                if cur and (len(cur) == L.SPLAT_MAX_SENSORS or cur_tiles + t > MAX_GROUP_TILES):
                    chunks.append(cur)
                    cur, cur_tiles = [], 0
                cur.append(item)
                cur_tiles += t
            if cur:
                chunks.append(cur)
            for chunk in chunks:
                fr = Frame([r[2] for _, r in chunk], scenes[sc]["means"].shape[0], self.C, self.device)
                self.groups.append((fr, sc, [(pos, j) for j, (pos, _) in enumerate(chunk)]))
        # size every group's intersection buffers once (a host read per group and round)
        for fr, sc, _ in self.groups:
            cg = fr.c_gaussians(scenes[sc])
            fr.project(cg)
            fr.bin_sort()
            need = int(fr.n_isect.item())
            while need > fr.capacity:
                fr._alloc_capacity(int(need * headroom) + 4096)
                fr.bin_sort()
                need = int(fr.n_isect.item())
        self.n = len(reqs)
        self.outputs = [None] * self.n
        self.requests = [None] * self.n
        c_reqs = (L.splat_batch_request * self.n)()
        for fr, sc, members in self.groups:
            g = scenes[sc]
            for pos, j in members:
                s = fr.sensors[j]
                R = s.n_rays
                out = {"feat": torch.empty((R, self.C), dtype=torch.float32, device=self.device),
                       "T": torch.empty(R, dtype=torch.float32, device=self.device)}
                if s.kind == "lidar":
                    for k in ("range_exp", "range_med", "alpha"):
                        out[k] = torch.empty(R, dtype=torch.float32, device=self.device)
                self.outputs[pos] = out
                self.requests[pos] = (reqs[pos][0], reqs[pos][1], s)
                c = c_reqs[pos]
                c.group_sensors = ctypes.cast(fr.c_sensors, ctypes.POINTER(L.splat_sensor))
                c.group_n_sensors = len(fr.sensors)
                c.group_sensor_index = j
                c.proj = fr.c_proj()
                c.bins = fr.c_bins()
                c.features = g["features"].data_ptr()
                c.n = fr.n
                c.channels = self.C
                c.out_feat = out["feat"].data_ptr()
                c.out_T = out["T"].data_ptr()
                if s.kind == "lidar":
                    c.out_range_exp = out["range_exp"].data_ptr()
                    c.out_range_med = out["range_med"].data_ptr()
                    c.out_alpha = out["alpha"].data_ptr()
        lib = L.load()
        nbytes = lib.splat_batch_table_bytes(self.n)
        host = (ctypes.c_uint8 * nbytes)()
        total = ctypes.c_int64()
        L.call("splat_batch_build", c_reqs, self.n, host, nbytes, ctypes.byref(total))
        self.total_items = total.value
        self.table = torch.frombuffer(bytearray(host), dtype=torch.uint8).to(self.device)
        self.counters = torch.zeros(self.n + 1, dtype=torch.int32, device=self.device)
        self.stamps = torch.zeros(self.n + 1, dtype=torch.int64, device=self.device)
        self.start = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.rays = sum(_rays(r[2]) for r in self.requests)
        self.graph = None

    def launches(self) -> int:
        """Kernels one batch launches (stamps, projections, sorts, the persistent launch)."""
        n = 1   # the start stamp
        for fr, _, _ in self.groups:
            bits = max(1, int(np.ceil(np.log2(max(fr.total_tiles, 2)))))
            passes = max(1, (bits + 7) // 8)
            # projection; binning: compaction scan, 4 depth passes (histogram, 3-launch
            # scan, scatter), row-item scan + rows, slot scan + slot totals, emission (with
            # the first tile pass's histogram), the tile passes, tile ranges
            n += 1 + (3 + 4 * 5 + 4 + 4 + 1 + passes * 5 - 1 + 1)
        return n + 2    # the persistent raster launch and its stamp

    def run(self):
        """One batch: the start stamp, every group's projection and binning (the groups are
        independent and spread over side streams, so that one group's short scan launches
        overlap another's), then the persistent raster launch over all requests."""
        cur = torch.cuda.current_stream()
        st = _stream(cur)
        L.call("splat_stamp", _vp(self.start), st)
        if not hasattr(self, "_side"):
            self._side = [torch.cuda.Stream(device=self.device) for _ in range(min(3, len(self.groups)))]
        for s in self._side:
            s.wait_stream(cur)
        for k, (fr, sc, _) in enumerate(self.groups):
            s = self._side[k % len(self._side)]
            cg = fr.c_gaussians(self.scenes[sc])
            fr.project(cg, stream=s)
            fr.bin_sort(stream=s)
        for s in self._side:
            cur.wait_stream(s)
        L.call("splat_render_batch", _vp(self.table), self.n, self.total_items, self.C, _vp(self.counters),
               _vp(self.stamps), None, st)

    def capture(self):
        torch.cuda.synchronize()
        self.run()                      # warm-up outside the capture (function attributes)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=s):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        return self

    def replay(self):
        self.graph.replay()

    def overflowed(self) -> bool:
        return any(int(fr.n_isect.item()) > fr.capacity for fr, _, _ in self.groups)

    def latencies_ms(self) -> np.ndarray:
        """Per-request completion time after the batch started (last replay), in ms."""
        st = self.stamps.cpu().numpy()
        t0 = int(self.start.item())
        return (st[:self.n] - t0) / 1e6

    def result(self, request_index: int) -> dict:
        """Outputs of the caller's request number `request_index`."""
        pos = self.order.index(request_index)
        return self.outputs[pos]


def stage_times(br: BatchRenderer, reps: int = 5) -> dict:
    """Where a batch's time goes: each stage launched on its own (eager, CUDA events,
    mean of `reps`) -- every group's projection, every group's binning, the persistent
    raster launch -- and the (ray, Gaussian) pairs the persistent launch examines
    (camera, lidar; its counting variant), the work behind its roofline.  When the
    batch's tile shapes are ones the per-frame kernels take, the same lists rasterized
    by the per-frame kernels (one camera and one lidar launch per group) are timed too."""
    stream = torch.cuda.current_stream()
    cgs = [fr.c_gaussians(br.scenes[sc]) for fr, sc, _ in br.groups]

    def timed(fn):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    def project():
        for (fr, _, _), cg in zip(br.groups, cgs):
            fr.project(cg)

    def binning():
        for fr, _, _ in br.groups:
            fr.bin_sort()

    def raster(ev=None):
        L.call("splat_render_batch", _vp(br.table), br.n, br.total_items, br.C, _vp(br.counters), _vp(br.stamps),
               _vp(ev), _stream())

    res = {"project": timed(project), "bin_sort": timed(binning), "persistent_raster": timed(raster)}
    ev = torch.zeros(2, dtype=torch.int64, device=br.device)
    raster(ev)
    torch.cuda.synchronize()
    res["evaluated_pairs"] = {"camera": int(ev[0].item()), "lidar": int(ev[1].item())}
    res["intersections"] = int(sum(int(fr.n_isect.item()) for fr, _, _ in br.groups))
    per_frame_ok = all(((s.tile_w, s.tile_h) in ((16, 16), (8, 8), (32, 8), (16, 32))) if s.kind == "camera" else
                       ((s.tile_az, s.tile_el) in ((32, 8), (16, 8), (32, 16), (64, 8)))
                       for fr, _, _ in br.groups for s in fr.sensors)
    res["per_frame_raster_same_lists"] = None
    if per_frame_ok:
        outs = [fr.alloc_outputs(False) for fr, _, _ in br.groups]

        def per_frame():
            for (fr, _, _), cg, o in zip(br.groups, cgs, outs):
                fr.rasterize(cg, o)
        res["per_frame_raster_same_lists"] = timed(per_frame)
        del outs
    return res


def time_replays(br: BatchRenderer, reps: int = 10):
    """Milliseconds per replay (CUDA events) and the per-request latencies of all replays."""
    stream = torch.cuda.current_stream()
    lat = []
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        br.replay()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        lat.append(br.latencies_ms())
    return np.array(times), np.concatenate(lat)


def autotune(scenes, requests, cam_shapes=None, lid_shapes=None, reps: int = 5, device="cuda", log=None):
    """Tries every (camera tile, lidar tile) pair of 256-ray shapes on the batch and
    returns (best BatchRenderer, table of ms per replay)."""
    cam_shapes = cam_shapes or CAMERA_SHAPES
    lid_shapes = lid_shapes or LIDAR_SHAPES
    results = {}
    best, best_ms = None, float("inf")
    for ct, lt in itertools.product(cam_shapes, lid_shapes):
        br = BatchRenderer(scenes, requests, ct, lt, device).capture()
        br.replay()
        ms, _ = time_replays(br, reps)
        results[(ct, lt)] = float(np.median(ms))
        if log:
            log(f"tiles camera {ct} lidar {lt}: {results[(ct, lt)]:.3f} ms")
        if results[(ct, lt)] < best_ms:
            if best is not None:
                del best
            best, best_ms = br, results[(ct, lt)]
        else:
            del br
        torch.cuda.empty_cache()
    return best, results
