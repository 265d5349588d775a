"""Small scene builders shared by the tests (inputs only, no renderer arithmetic)."""
import math

import numpy as np

from paper_2411_16816_gb300 import scenes


def one_gaussian(mean, scale, quat=(1.0, 0.0, 0.0, 0.0), opacity=0.9, feature=(1.0,), vel=(0.0, 0.0, 0.0),
                 dtype=np.float64):
    return {
        "means": np.asarray([mean], dtype=dtype), "scales": np.asarray([scale], dtype=dtype),
        "quats": np.asarray([quat], dtype=dtype), "opacities": np.asarray([opacity], dtype=dtype),
        "features": np.asarray([feature], dtype=dtype), "velocities": np.asarray([vel], dtype=dtype),
    }


def stack(*gs):
    return {k: np.concatenate([g[k] for g in gs]) for k in gs[0]}


def empty_scene(channels=3):
    return {"means": np.zeros((0, 3), np.float32), "scales": np.zeros((0, 3), np.float32),
            "quats": np.zeros((0, 4), np.float32), "opacities": np.zeros(0, np.float32),
            "features": np.zeros((0, channels), np.float32), "velocities": np.zeros((0, 3), np.float32)}


def front_camera(width=128, height=96, f=100.0, **kw):
    return scenes.Camera(R=scenes.camera_rotation(0.0), t=np.zeros(3), width=width, height=height,
                         fx=f, fy=f, cx=width / 2, cy=height / 2, **kw)


def small_lidar(n_beams=16, n_az=256, lo=-15.0, hi=15.0, **kw):
    elev = np.deg2rad(np.linspace(lo, hi, n_beams))
    az_res = 2 * math.pi / n_az
    kw.setdefault("eps2d", scenes.lidar_blur(elev, az_res))
    kw.setdefault("R", np.eye(3))
    kw.setdefault("t", np.zeros(3))
    return scenes.Lidar(beam_elev=elev, n_az=n_az, az_res=az_res, **kw)


def rodrigues(axis_angle):
    """Rotation matrix of an axis-angle vector (textbook Rodrigues formula)."""
    v = np.asarray(axis_angle, dtype=np.float64)
    th = np.linalg.norm(v)
    if th == 0:
        return np.eye(3)
    k = v / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def random_small_scene(seed, n, box_lo, box_hi, channels, log_scale=(-1.0, 0.3), dynamic=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return {
        "means": rng.uniform(box_lo, box_hi, size=(n, 3)),
        "scales": np.exp(rng.normal(log_scale[0], log_scale[1], size=(n, 3))),
        "quats": q * rng.uniform(0.5, 2.0, size=(n, 1)),
        "opacities": rng.uniform(0.2, 0.95, size=n),
        "features": rng.normal(size=(n, channels)),
        "velocities": rng.normal(0, 1.5, size=(n, 3)) if dynamic else np.zeros((n, 3)),
    }
