"""Seeded synthetic scenes and sensor rigs shaped like driving logs.

This module only draws inputs: Gaussian parameters, sensor poses, intrinsics
and lidar beam layouts. It holds none of the renderer's arithmetic (no
projection, tiling, blending or gradients), so that the FP64 oracle and the
CUDA library can both consume the very same arrays without sharing code.

Conventions (world frame): x forward, y left, z up; every sensor sits at the
origin at its mid-capture time.  Camera frame: z forward, x right, y down.
Lidar frame: x forward, y left, z up.  Poses are world->sensor rotations R
(row-major 3x3) and translations t, so a world point p maps to R p + t.
Sensor linear/angular velocities are expressed in the sensor frame.

All random draws use numpy ``Generator(PCG64(seed))`` in FP64 and are cast to
FP32 once.  Quaternions are w-x-y-z, drawn as normalised 4-D normals (uniform
on S^3).  Scales are returned already exponentiated and opacities already
passed through a logistic sigmoid (the library takes activated values).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def random_gaussians(n: int, seed: int, lo, hi, log_scale_mu: float, log_scale_sd: float,
                     channels: int, feature_dist: str = "uniform", dynamic_frac: float = 0.0,
                     vel_sd: float = 0.0, min_radius: float = 0.0) -> dict:
    """Draw ``n`` Gaussians with means uniform in the box [lo, hi].

    ``min_radius`` > 0 rejects means whose horizontal distance to the origin
    is below it (the ego vehicle's own footprint holds no scene content).
    Returns FP32 arrays: means (n,3), scales (n,3), quats (n,4), opacities
    (n,), features (n,channels), velocities (n,3).
    """
    rng = _rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    means = rng.uniform(lo, hi, size=(n, 3))
    if min_radius > 0.0 and n > 0:
        bad = np.hypot(means[:, 0], means[:, 1]) < min_radius
        while bad.any():
            means[bad] = rng.uniform(lo, hi, size=(int(bad.sum()), 3))
            bad = np.hypot(means[:, 0], means[:, 1]) < min_radius
    scales = np.exp(rng.normal(log_scale_mu, log_scale_sd, size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = _sigmoid(rng.normal(size=n))
    if feature_dist == "uniform":
        feats = rng.uniform(0.0, 1.0, size=(n, channels))
    else:
        feats = rng.normal(size=(n, channels))
    vel = np.zeros((n, 3))
    if dynamic_frac > 0.0 and n > 0:
        dyn = rng.uniform(size=n) < dynamic_frac
        vel[dyn] = rng.normal(0.0, vel_sd, size=(int(dyn.sum()), 3))
    return {
        "means": means.astype(F32), "scales": scales.astype(F32), "quats": q.astype(F32),
        "opacities": opac.astype(F32), "features": np.ascontiguousarray(feats.astype(F32)),
        "velocities": vel.astype(F32),
    }


def yaw_matrix(yaw: float) -> np.ndarray:
    """Rotation (world) about +z by ``yaw`` radians."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def camera_rotation(yaw: float) -> np.ndarray:
    """World->camera rotation for a level camera looking along heading ``yaw``.

    Rows are the camera axes written in world coordinates: right, down, forward.
    """
    c, s = math.cos(yaw), math.sin(yaw)
    fwd = np.array([c, s, 0.0])
    right = np.array([s, -c, 0.0])
    down = np.array([0.0, 0.0, -1.0])
    return np.stack([right, down, fwd])


@dataclass
class Camera:
    R: np.ndarray
    t: np.ndarray
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    lin_vel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    ang_vel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    rs_time: float = 0.0
    time_offset: float = 0.0
    eps2d: float = 0.3
    near: float = 0.01
    tile_w: int = 16
    tile_h: int = 16
    support: int = 0               # tile extent flags: 1 opacity-aware, 2 lidar sweep-time margins
    kind: str = "camera"

    @property
    def n_rays(self) -> int:
        return self.width * self.height


@dataclass
class Lidar:
    R: np.ndarray
    t: np.ndarray
    beam_elev: np.ndarray          # (n_beams,) radians, ascending
    n_az: int
    az_res: float                  # radians per azimuth bin
    sweep_time: float = 0.0
    eps2d: float = 0.0             # blur added to the (phi, omega) covariance, rad^2
    r_min: float = 0.1
    lin_vel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    ang_vel: np.ndarray = field(default_factory=lambda: np.zeros(3))
    tile_az: int = 32
    tile_el: int = 8
    rays: np.ndarray | None = None  # optional (n_beams, n_az, 3) of (phi, omega, t)
    support: int = 0               # tile extent flags: 1 opacity-aware, 2 lidar sweep-time margins
    kind: str = "lidar"

    @property
    def n_beams(self) -> int:
        return int(len(self.beam_elev))

    @property
    def n_rays(self) -> int:
        return self.n_beams * self.n_az


def lidar_blur(beam_elev: np.ndarray, az_res: float, factor: float = 0.3) -> float:
    """Blur term for a lidar: ``factor`` x (azimuth step x mean elevation step).

    This is the lidar counterpart of 0.3 px^2 per pixel area; it is an input
    parameter of the renderer, chosen here from the beam layout.
    """
    el = np.asarray(beam_elev, dtype=np.float64)
    d_el = (el[-1] - el[0]) / max(len(el) - 1, 1)
    return float(factor * az_res * d_el)


def nonuniform_elevations(n_beams: int, lo_deg: float = -25.0, hi_deg: float = 15.0,
                          split: float = 0.625) -> np.ndarray:
    """Beam elevations denser near the horizon (spacing grows as |u-split|^0.5)."""
    u = (np.arange(n_beams) + 0.5) / n_beams
    d = u - split
    up = hi_deg * (np.clip(d, 0, None) / (1.0 - split)) ** 1.5
    dn = lo_deg * (np.clip(-d, 0, None) / split) ** 1.5
    return np.deg2rad(np.where(d >= 0, up, dn))


def ego_motion(R: np.ndarray, speed: float, yaw_rate: float):
    """Sensor-frame linear and angular velocity of a rig moving along world +x."""
    v_world = np.array([speed, 0.0, 0.0])
    w_world = np.array([0.0, 0.0, yaw_rate])
    return R @ v_world, R @ w_world


# ----------------------------------------------------------------------------
# The five workloads.  Config k uses seed 1000 + k; targets use seed + 1.
# ----------------------------------------------------------------------------

def tiny_frame(seed: int = 1001, n: int = 2000):
    """2,000 Gaussians 5-25 m ahead; one 128x96 camera (f=100) and a 16x256 lidar."""
    g = random_gaussians(n, seed, lo=(5.0, -10.0, -10.0), hi=(25.0, 10.0, 10.0),
                         log_scale_mu=-2.0, log_scale_sd=0.5, channels=3, feature_dist="uniform")
    cam = Camera(R=camera_rotation(0.0), t=np.zeros(3), width=128, height=96,
                 fx=100.0, fy=100.0, cx=64.0, cy=48.0)
    elev = np.deg2rad(np.linspace(-15.0, 15.0, 16))
    az_res = 2.0 * math.pi / 256
    lid = Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=256, az_res=az_res,
                eps2d=lidar_blur(elev, az_res))
    return g, [cam, lid]


def driving_rig(speed: float = 15.0, yaw_rate: float = 0.05, width: int = 1920, height: int = 1080,
                n_cams: int = 6, n_beams: int = 32, n_az: int = 1080, rs_time: float = 0.03,
                sweep_time: float = 0.1):
    """Six 60-degree ring cameras with rolling shutter and one spinning lidar."""
    sensors = []
    f = (width / 2) / math.tan(math.radians(30.0))
    for k in range(n_cams):
        R = camera_rotation(k * math.pi / 3)
        v, w = ego_motion(R, speed, yaw_rate)
        sensors.append(Camera(R=R, t=np.zeros(3), width=width, height=height, fx=f, fy=f,
                              cx=width / 2, cy=height / 2, lin_vel=v, ang_vel=w, rs_time=rs_time))
    elev = np.deg2rad(np.linspace(-25.0, 15.0, n_beams))
    az_res = 2.0 * math.pi / n_az
    v, w = ego_motion(np.eye(3), speed, yaw_rate)
    sensors.append(Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=n_az, az_res=az_res,
                         sweep_time=sweep_time, eps2d=lidar_blur(elev, az_res), lin_vel=v, ang_vel=w))
    return sensors


def driving_gaussians(n: int, seed: int, channels: int = 16, min_radius: float = 2.0):
    """Driving-scale scene: 100x100x10 m box, 20% dynamic Gaussians (sd 2 m/s)."""
    return random_gaussians(n, seed, lo=(-50.0, -50.0, -2.0), hi=(50.0, 50.0, 8.0),
                            log_scale_mu=-1.5, log_scale_sd=0.7, channels=channels,
                            feature_dist="normal", dynamic_frac=0.2, vel_sd=2.0,
                            min_radius=min_radius)


def driving_frame(seed: int = 1002, n: int = 500_000, **rig):
    """500k Gaussians, six 1920x1080 rolling-shutter cameras, 32x1080 lidar."""
    return driving_gaussians(n, seed), driving_rig(**rig)


def lidar_heavy_frame(seed: int = 1003, n: int = 1_000_000, channels: int = 16):
    """1M Gaussians and a 128-beam x 2048 non-uniform lidar, 100 ms sweep at 15 m/s."""
    g = driving_gaussians(n, seed, channels=channels)
    elev = nonuniform_elevations(128)
    az_res = 2.0 * math.pi / 2048
    v, w = ego_motion(np.eye(3), 15.0, 0.0)
    lid = Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=2048, az_res=az_res,
                sweep_time=0.1, eps2d=lidar_blur(elev, az_res), lin_vel=v, ang_vel=w)
    return g, [lid]


def target_like(g: dict, seed: int) -> dict:
    """Same geometry with re-drawn features and opacities (an L1 target scene)."""
    rng = _rng(seed)
    out = dict(g)
    n, c = g["features"].shape
    out["features"] = rng.normal(size=(n, c)).astype(F32)
    out["opacities"] = _sigmoid(rng.normal(size=n)).astype(F32)
    return out


def subset(g: dict, idx) -> dict:
    return {k: np.ascontiguousarray(v[idx]) for k, v in g.items()}


# ----------------------------------------------------------------------------------------
# Learned ray head inputs: initial weights and a seeded ground-truth "teacher"
# ----------------------------------------------------------------------------------------

HEAD_SHAPES = {"W1": (32, 64), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (64, 2), "b3": (2,)}
HEAD_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def head_init_params(seed: int) -> dict:
    """Seeded initial weights of the 32 -> 64 -> 64 -> 2 head (uniform, fan-in scaled; zero
    biases), FP32 masters."""
    rng = _rng(seed)
    p = {}
    for k in HEAD_ORDER:
        shape = HEAD_SHAPES[k]
        if len(shape) == 2:
            b = 1.0 / math.sqrt(shape[0])
            p[k] = rng.uniform(-b, b, size=shape).astype(F32)
        else:
            p[k] = np.zeros(shape, F32)
    return p


def teacher_params(seed: int, n_feat: int = 29) -> dict:
    """A frozen random network that defines the synthetic lidar ground truth: its two
    outputs depend non-linearly on the rendered features and on the ray direction, so a
    view-independent per-Gaussian channel cannot reproduce them."""
    rng = _rng(seed)
    return {"A": rng.normal(0, 1.0 / math.sqrt(n_feat + 3), size=(n_feat + 3, 24)),
            "a": rng.normal(0, 0.3, size=24),
            "B": rng.normal(0, 1.2 / math.sqrt(24), size=(24, 2)),
            "D": rng.normal(0, 1.0, size=(3, 2)), "c": np.array([0.2, -0.8])}


def teacher_labels(feat: np.ndarray, dirs: np.ndarray, tp: dict, seed: int):
    """Ground-truth intensity in [0, 1] and Bernoulli ray-drop labels for rays with
    rendered features `feat` (R x F) and unit directions `dirs` (R x 3)."""
    x = np.concatenate([feat, dirs], axis=1).astype(np.float64)
    h = np.tanh(x @ tp["A"] + tp["a"])
    z = h @ tp["B"] + (dirs ** 2) @ tp["D"] + tp["c"]
    intensity = 1.0 / (1.0 + np.exp(-z[:, 0]))
    p_drop = 1.0 / (1.0 + np.exp(-z[:, 1]))
    drop = (_rng(seed).uniform(size=len(p_drop)) < p_drop).astype(F32)
    return intensity.astype(F32), drop, p_drop.astype(F32)



# ----------------------------------------------------------------------------------------
# Serving batch: 64 mixed requests over three scenes
# ----------------------------------------------------------------------------------------

def serving_batch(seed: int = 1005, sizes=(200_000, 800_000, 2_000_000), channels: int = 16):
    """Three driving scenes (200k / 800k / 2M Gaussians) and 64 requests assigned to them
    round-robin: 12 x 640x480, 12 x 1280x720, 12 x 1920x1080 rolling-shutter cameras (60-
    degree field of view), 14 x 32-beam x 1080 and 14 x 128-beam x 2048 lidar sweeps, each
    at a random heading of a rig moving at 15 m/s.  Returns (scenes, [(scene, sensor)])."""
    rng = _rng(seed)
    scene_list = [driving_gaussians(n, seed + 10 * k, channels=channels) for k, n in enumerate(sizes)]
    kinds = ([("cam", 640, 480)] * 12 + [("cam", 1280, 720)] * 12 + [("cam", 1920, 1080)] * 12 +
             [("lid", 32, 1080)] * 14 + [("lid", 128, 2048)] * 14)
    requests = []
    for q, kind in enumerate(kinds):
        yaw = float(rng.uniform(0, 2 * math.pi))
        if kind[0] == "cam":
            w, h = kind[1], kind[2]
            R = camera_rotation(yaw)
            v, om = ego_motion(R, 15.0, 0.05)
            f = (w / 2) / math.tan(math.radians(30.0))
            s = Camera(R=R, t=np.zeros(3), width=w, height=h, fx=f, fy=f, cx=w / 2, cy=h / 2, lin_vel=v,
                       ang_vel=om, rs_time=0.03)
        else:
            nb, naz = kind[1], kind[2]
            elev = np.deg2rad(np.linspace(-25.0, 15.0, nb)) if nb == 32 else nonuniform_elevations(nb)
            R = yaw_matrix(yaw).T
            v, om = ego_motion(R, 15.0, 0.05)
            res = 2 * math.pi / naz
            s = Lidar(R=R, t=np.zeros(3), beam_elev=elev, n_az=naz, az_res=res, sweep_time=0.1,
                      eps2d=lidar_blur(elev, res), lin_vel=v, ang_vel=om)
        requests.append((q % len(sizes), s))
    return scene_list, requests
