"""Batched serving: one persistent, graph-captured launch over many cameras and lidar
sweeps of several scenes must reproduce the per-frame path exactly and the oracle
within the parity tolerances, whatever 256-ray tile shape each sensor kind uses."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_16816_gb300 import scenes
from paper_2411_16816_gb300.batch import BatchRenderer, autotune, time_replays
from paper_2411_16816_gb300.render import gaussians_to_device
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _small_batch(seed=7):
    rng = np.random.default_rng(seed)
    sc = [scenes.random_gaussians(n, seed + k, lo=(-25, -25, -2), hi=(25, 25, 8), log_scale_mu=-1.3,
                                  log_scale_sd=0.5, channels=16, feature_dist="normal", dynamic_frac=0.2, vel_sd=2.0,
                                  min_radius=2.0) for k, n in enumerate((6000, 15000))]
    reqs = []
    for q, (w, h) in enumerate([(160, 120), (320, 240), (200, 100), (96, 64), (320, 180), (150, 90)]):
        yaw = float(rng.uniform(0, 2 * math.pi))
        R = scenes.camera_rotation(yaw)
        v, om = scenes.ego_motion(R, 15.0, 0.05)
        f = (w / 2) / math.tan(math.radians(30.0))
        reqs.append((q % 2, scenes.Camera(R=R, t=np.zeros(3), width=w, height=h, fx=f, fy=f, cx=w / 2, cy=h / 2,
                                          lin_vel=v, ang_vel=om, rs_time=0.03)))
    for q, (nb, naz) in enumerate([(32, 512), (64, 1024), (32, 1080), (16, 256)]):
        yaw = float(rng.uniform(0, 2 * math.pi))
        R = scenes.yaw_matrix(yaw).T
        v, om = scenes.ego_motion(R, 15.0, 0.05)
        elev = scenes.nonuniform_elevations(nb)
        res = 2 * math.pi / naz
        reqs.append((q % 2, scenes.Lidar(R=R, t=np.zeros(3), beam_elev=elev, n_az=naz, az_res=res, sweep_time=0.1,
                                         eps2d=scenes.lidar_blur(elev, res), lin_vel=v, ang_vel=om)))
    return sc, reqs


def _views(br, pos):
    req_idx, sc, s = br.requests[pos]
    return req_idx, sc, s, br.outputs[pos]


def test_batch_equals_per_frame_path_bitwise():
    sc, reqs = _small_batch()
    gd = [gaussians_to_device(g, DEV) for g in sc]
    br = BatchRenderer(gd, reqs, (16, 16), (32, 8), DEV).capture()
    br.replay()
    torch.cuda.synchronize()
    assert not br.overflowed()
    for fr, si, members in br.groups:
        out = fr.alloc_outputs(keep_state=True)
        fr.rasterize(fr.c_gaussians(gd[si]), out)
        torch.cuda.synchronize()
        cams = fr.split(out["cam_feat"], "camera") if fr.cam_idx else []
        lids = fr.split(out["lid_feat"], "lidar") if fr.lid_idx else []
        rng_l = fr.split(out["lid_range_exp"], "lidar") if fr.lid_idx else []
        for pos, j in members:
            s = fr.sensors[j]
            o = br.outputs[pos]
            if s.kind == "camera":
                ref = cams[fr.cam_idx.index(j)].reshape(-1, 16)
                assert torch.equal(o["feat"], ref)
            else:
                k = fr.lid_idx.index(j)
                assert torch.equal(o["feat"], lids[k].reshape(-1, 16))
                assert torch.equal(o["range_exp"], rng_l[k].reshape(-1))


@pytest.mark.parametrize("cam_tile, lid_tile", [((8, 32), (16, 16)), ((64, 4), (64, 4))])
def test_batch_matches_oracle_with_other_tile_shapes(cam_tile, lid_tile):
    sc, reqs = _small_batch(seed=9)
    gd = [gaussians_to_device(g, DEV) for g in sc]
    br = BatchRenderer(gd, reqs, cam_tile, lid_tile, DEV).capture()
    br.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for pos in range(br.n):
        req_idx, si, s, o = _views(br, pos)
        sel = np.sort(rng.choice(s.n_rays, size=min(96, s.n_rays), replace=False))
        ref = oracle.render_variants(sc[si], s, sel=sel)
        got = {"F": o["feat"].cpu().numpy()[sel]}
        if s.kind == "lidar":
            got["range_exp"] = o["range_exp"].cpu().numpy()[sel]
        U.check_variants(s.kind, got, ref, what=f"request {req_idx}")


def test_replays_are_deterministic_and_stamped():
    sc, reqs = _small_batch(seed=11)
    gd = [gaussians_to_device(g, DEV) for g in sc]
    br = BatchRenderer(gd, reqs, (32, 8), (32, 8), DEV).capture()
    br.replay()
    torch.cuda.synchronize()
    first = [o["feat"].clone() for o in br.outputs]
    ms, lat = time_replays(br, reps=3)
    for a, o in zip(first, br.outputs):
        assert torch.equal(a, o["feat"])
    assert (lat > 0).all() and (lat <= ms.max() * 1.5 + 1.0).all()


def test_autotuner_picks_a_tiling():
    sc, reqs = _small_batch(seed=13)
    gd = [gaussians_to_device(g, DEV) for g in sc]
    best, table = autotune(gd, reqs, cam_shapes=[(16, 16), (32, 8)], lid_shapes=[(32, 8), (16, 16)], reps=2)
    assert len(table) == 4 and all(v > 0 for v in table.values())
    best.replay()
    torch.cuda.synchronize()
    assert not best.overflowed()


def test_batch_work_counter_equals_the_per_frame_counts():
    """The persistent launch's counting variant examines exactly the (ray, Gaussian) pairs
    the per-frame kernels examine on the same lists (camera and lidar separately), and the
    stage breakdown covers every stage."""
    from paper_2411_16816_gb300.batch import stage_times
    sc, reqs = _small_batch(seed=17)
    gd = [gaussians_to_device(g, DEV) for g in sc]
    br = BatchRenderer(gd, reqs, (16, 16), (32, 8), DEV).capture()
    br.replay()
    want = torch.zeros(2, dtype=torch.int64, device=DEV)
    for fr, si, _ in br.groups:
        fr.rasterize(fr.c_gaussians(gd[si]), fr.alloc_outputs(False), evaluated=want)
    st = stage_times(br, reps=2)
    torch.cuda.synchronize()
    assert st["evaluated_pairs"]["camera"] == int(want[0]) > 0
    assert st["evaluated_pairs"]["lidar"] == int(want[1]) > 0
    for k in ("project", "bin_sort", "persistent_raster", "per_frame_raster_same_lists"):
        assert st[k] > 0, k
