"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's general formulas: expected values come from
closed forms of special geometries, finite differences of the plain projection
maps, brute-force enumeration, or invariants.  The paper prints no worked
numerical example, so there are no golden values from the paper itself.
"""
import math

import numpy as np
import pytest

import oracle
from tests.helpers import (empty_scene, front_camera, one_gaussian, quat_mul, random_small_scene, rodrigues,
                           small_lidar, stack)
from paper_2411_16816_gb300 import scenes

A_MIN = 1.0 / 255.0
EPS = float(np.float32(0.3))   # the camera blur, as the library receives it (FP32)


# ----------------------------------------------------------------------------------
# Projection closed forms (Sec. 3.2): Gaussian on the optical axis
# ----------------------------------------------------------------------------------

def test_camera_axis_aligned_covariance_closed_form():
    cam = front_camera(f=100.0)
    z, sx, sy, sz = 12.0, 0.3, 0.5, 0.2
    g = one_gaussian((z, 0.0, 0.0), (sx, sy, sz), opacity=0.8)
    p = oracle.project(g, cam)
    rec = p["rec"][0]
    # camera x = -world y, camera y = -world z, camera z = world x, J = diag(f/z) on the axis
    k = (cam.fx / z) ** 2
    A, C = k * sy * sy + EPS, k * sz * sz + EPS
    assert rec[0] == pytest.approx(cam.cx, abs=1e-12) and rec[1] == pytest.approx(cam.cy, abs=1e-12)
    assert rec[10] == pytest.approx(A, rel=1e-12) and rec[12] == pytest.approx(C, rel=1e-12)
    assert abs(rec[11]) < 1e-12
    comp = math.sqrt((A - EPS) * (C - EPS) / (A * C))
    assert rec[13] == pytest.approx(comp, rel=1e-12)
    assert rec[5] == pytest.approx(0.8 * comp, rel=1e-12)
    assert rec[2] == pytest.approx(1 / A, rel=1e-12) and rec[4] == pytest.approx(1 / C, rel=1e-12)
    assert rec[6] == pytest.approx(z, rel=1e-12)


@pytest.mark.parametrize("q, perm", [
    ((math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)), (1, 0, 2)),   # 90 deg about z: world cov diag(sy,sx,sz)
    ((math.cos(math.pi / 4), math.sin(math.pi / 4), 0, 0), (0, 2, 1)),   # 90 deg about x: diag(sx,sz,sy)
])
def test_camera_quaternion_rotates_covariance(q, perm):
    cam = front_camera(f=100.0)
    z, s = 10.0, np.array([0.2, 0.45, 0.7])
    g = one_gaussian((z, 0, 0), s, quat=q)
    rec = oracle.project(g, cam)["rec"][0]
    sw = s[list(perm)]       # world-axis standard deviations after the rotation
    k = (cam.fx / z) ** 2
    # image x <- world y, image y <- world z
    assert rec[10] == pytest.approx(k * sw[1] ** 2 + EPS, rel=1e-10)
    assert rec[12] == pytest.approx(k * sw[2] ** 2 + EPS, rel=1e-10)
    assert abs(rec[11]) < 1e-9


@pytest.mark.parametrize("yaw", [0.0, 0.7, -2.1])
def test_camera_off_axis_mean(yaw):
    cam = scenes.Camera(R=scenes.camera_rotation(yaw), t=np.zeros(3), width=200, height=100, fx=120, fy=90,
                        cx=101.5, cy=47.0)
    fwd = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.array([0.0, 0.0, -1.0])
    d, a, b = 9.0, 1.3, -0.6
    g = one_gaussian(d * fwd + a * right + b * down, (0.1, 0.1, 0.1))
    rec = oracle.project(g, cam)["rec"][0]
    # the rotation reaches the renderer rounded to FP32: agreement to ~1e-7 relative
    assert rec[0] == pytest.approx(101.5 + 120 * a / d, rel=1e-6)
    assert rec[1] == pytest.approx(47.0 + 90 * b / d, rel=1e-6)
    assert rec[6] == pytest.approx(d, rel=1e-6)


# ----------------------------------------------------------------------------------
# Jacobians vs finite differences of the plain maps
# ----------------------------------------------------------------------------------

def _fd_jac(fun, x, h=1e-6):
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for k in range(len(x)):
        e = np.zeros_like(x)
        e[k] = h
        cols.append((np.asarray(fun(x + e)) - np.asarray(fun(x - e))) / (2 * h))
    return np.stack(cols, axis=1)


def test_camera_jacobian_and_covariance_match_fd():
    cam = scenes.Camera(R=scenes.camera_rotation(0.3), t=np.array([0.2, -0.1, 0.5]), width=160, height=120,
                        fx=110, fy=95, cx=80, cy=60)
    rng = np.random.default_rng(5)
    for _ in range(5):
        mean = np.array([8.0, 2.0, 0.5]) + rng.normal(0, 0.5, 3)
        scale = np.exp(rng.normal(-1, 0.3, 3))
        q = rng.normal(size=4)
        vis, J, Sc, _ = oracle.jacobian(mean, scale, q, 0.9, cam)
        assert vis
        m = np.asarray(cam.R, dtype=np.float32).astype(np.float64) @ np.asarray(mean, np.float32) + \
            np.asarray(cam.t, np.float32)
        proj = lambda p: np.array([np.float32(110) * p[0] / p[2], np.float32(95) * p[1] / p[2]])
        Jfd = _fd_jac(proj, m)
        np.testing.assert_allclose(J[:2], Jfd, rtol=1e-6, atol=1e-8)
        rec = oracle.project(one_gaussian(np.float32(mean), np.float32(scale), np.float32(q)), cam)["rec"][0]
        S2 = Jfd @ Sc @ Jfd.T + EPS * np.eye(2)
        np.testing.assert_allclose([rec[10], rec[11], rec[12]], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6,
                                   atol=1e-7 * np.abs(S2).max())


def test_lidar_jacobian_matches_fd_all_rows():
    lid = small_lidar(R=rodrigues([0.1, -0.2, 0.4]))
    rng = np.random.default_rng(9)
    sph = lambda p: np.array([math.atan2(p[1], p[0]), math.asin(p[2] / np.linalg.norm(p)), np.linalg.norm(p)])
    for _ in range(6):
        mean = rng.normal(0, 6, 3)
        vis, J, Sc, _ = oracle.jacobian(mean, (0.3, 0.2, 0.1), (1, 0, 0, 0), 0.9, lid)
        m = np.asarray(lid.R, np.float32).astype(np.float64) @ np.asarray(mean, np.float32)
        np.testing.assert_allclose(J, _fd_jac(sph, m), rtol=1e-6, atol=1e-9)


def _exact_motion(m0, R, vs, ws, vg, t):
    """Sensor-frame position of a point at time t: the sensor translates with vs and
    rotates with ws (its own frame) while the point moves with world velocity vg."""
    return rodrigues(-np.asarray(ws) * t) @ (m0 + (R @ vg - vs) * t)


def test_pixel_velocity_matches_reprojection_fd():
    R = scenes.camera_rotation(0.4)
    vs, ws = np.array([0.5, -0.2, 14.0]), np.array([0.02, 0.06, -0.01])
    cam = scenes.Camera(R=R, t=np.zeros(3), width=200, height=150, fx=150, fy=150, cx=100, cy=75,
                        lin_vel=vs, ang_vel=ws, rs_time=0.03)
    R32 = np.asarray(R, np.float32).astype(np.float64)
    vs32, ws32 = np.asarray(vs, np.float32).astype(np.float64), np.asarray(ws, np.float32).astype(np.float64)
    for mean, vg in [((10.0, 5.0, 0.3), (0.0, 0.0, 0.0)), ((12.0, 4.0, -1.0), (1.5, -2.0, 0.4))]:
        g = one_gaussian(np.float32(mean), (0.2, 0.2, 0.2), vel=np.float32(vg))
        rec = oracle.project(g, cam)["rec"][0]
        m0 = R32 @ np.asarray(mean, np.float32)
        vg32 = np.asarray(vg, np.float32).astype(np.float64)
        pix = lambda t: (lambda p: np.array([150 * p[0] / p[2] + 100, 150 * p[1] / p[2] + 75]))(
            _exact_motion(m0, R32, vs32, ws32, vg32, t))
        h = 1e-5
        v_fd = (pix(h) - pix(-h)) / (2 * h)
        np.testing.assert_allclose(rec[7:9], v_fd, rtol=1e-6, atol=1e-6)


def test_lidar_velocity_matches_reprojection_fd():
    R = rodrigues([0.0, 0.0, 0.3])
    vs, ws = np.array([15.0, 0.5, 0.0]), np.array([0.0, 0.01, 0.05])
    lid = small_lidar(R=R, lin_vel=vs, ang_vel=ws, sweep_time=0.1)
    R32 = np.asarray(R, np.float32).astype(np.float64)
    vs32, ws32 = np.asarray(vs, np.float32).astype(np.float64), np.asarray(ws, np.float32).astype(np.float64)
    mean, vg = (6.0, -9.0, 1.0), (2.0, 1.0, -0.5)
    g = one_gaussian(np.float32(mean), (0.2, 0.2, 0.2), vel=np.float32(vg))
    rec = oracle.project(g, lid)["rec"][0]
    m0 = R32 @ np.asarray(mean, np.float32)
    vg32 = np.asarray(vg, np.float32).astype(np.float64)
    sph = lambda p: np.array([math.atan2(p[1], p[0]), math.asin(p[2] / np.linalg.norm(p)), np.linalg.norm(p)])
    f = lambda t: sph(_exact_motion(m0, R32, vs32, ws32, vg32, t))
    h = 1e-5
    np.testing.assert_allclose(rec[7:10], (f(h) - f(-h)) / (2 * h), rtol=1e-6, atol=1e-7)


# ----------------------------------------------------------------------------------
# Single-Gaussian renders in closed form (Eq. alpha, alpha blend, delta)
# ----------------------------------------------------------------------------------

def test_camera_single_gaussian_closed_form_render():
    cam = front_camera(width=64, height=48, f=60.0)
    z, sy, sz, o, f = 6.0, 0.35, 0.25, 0.85, 0.7
    g = one_gaussian((z, 0.2, -0.1), (0.3, sy, sz), opacity=o, feature=(f, 2 * f, -f))
    r = oracle.render(g, cam)
    # on-axis approximation does not hold off-axis, so use the exact affine footprint:
    # mean in pixels and the covariance from the physical geometry at (x, y, z)
    x, y = -0.2, 0.1            # camera-frame offsets (right = -world y, down = -world z)
    mu = np.array([60 * x / z + 32, 60 * y / z + 24])
    J = np.array([[60 / z, 0, -60 * x / z ** 2], [0, 60 / z, -60 * y / z ** 2]])
    Sc = np.diag([sy ** 2, sz ** 2, 0.3 ** 2])
    S2 = J @ Sc @ J.T + EPS * np.eye(2)
    comp = math.sqrt(np.linalg.det(S2 - EPS * np.eye(2)) / np.linalg.det(S2))
    inv = np.linalg.inv(S2)
    cols, rows = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    d = np.stack([cols - mu[0], rows - mu[1]], -1)
    alpha = np.minimum(o * comp * np.exp(-0.5 * np.einsum("...i,ij,...j->...", d, inv, d)), 0.999)
    # tiles intersected by the 3-sigma box
    ex, ey = 3 * math.sqrt(S2[0, 0]), 3 * math.sqrt(S2[1, 1])
    tx, ty = np.floor((cols - 0.5) / 16), np.floor((rows - 0.5) / 16)
    inside = ((tx + 1) * 16 > mu[0] - ex) & (tx * 16 < mu[0] + ex) & ((ty + 1) * 16 > mu[1] - ey) & (ty * 16 < mu[1] + ey)
    alpha = np.where(inside & (alpha >= A_MIN), alpha, 0.0).reshape(-1)
    assert alpha.max() > 0.5
    np.testing.assert_allclose(r["F"][:, 0], f * alpha, atol=1e-12)
    np.testing.assert_allclose(r["F"][:, 1], 2 * f * alpha, atol=1e-12)
    np.testing.assert_allclose(r["T"], 1 - alpha, atol=1e-12)


def test_lidar_single_gaussian_straddling_zero_azimuth():
    lid = small_lidar()
    r0, o = 10.0, 0.9
    sy, sz = 0.4, 0.3
    g = one_gaussian((r0, 0.0, 0.0), (0.3, sy, sz), opacity=o, feature=(1.0, -2.0))
    out = oracle.render(g, lid)
    el = np.asarray(lid.beam_elev, np.float32).astype(np.float64)
    res = float(np.float32(lid.az_res))
    eps = float(np.float32(lid.eps2d))
    # at (r,0,0): d(phi)/dy = 1/r, d(omega)/dz = 1/r -> diagonal spherical covariance
    A, C = (sy / r0) ** 2 + eps, (sz / r0) ** 2 + eps
    comp = math.sqrt((A - eps) * (C - eps) / (A * C))
    phi = (np.arange(256) + 0.5) * res
    dphi = np.where(phi > math.pi, phi - 2 * math.pi, phi)
    om = el[:, None]
    alpha = o * comp * np.exp(-0.5 * (dphi[None, :] ** 2 / A + om ** 2 / C))
    alpha = np.minimum(alpha, 0.999)
    cols = np.arange(256) // 32
    alpha = np.where((cols[None, :] == 0) | (cols[None, :] == 7), alpha, 0.0)
    alpha = np.where(alpha >= A_MIN, alpha, 0.0).reshape(-1)
    assert alpha.max() > 0.5 and (alpha[np.arange(4096) % 256 >= 224] > 0).any()
    np.testing.assert_allclose(out["F"][:, 0], alpha, atol=1e-12)
    np.testing.assert_allclose(out["F"][:, 1], -2 * alpha, atol=1e-12)
    np.testing.assert_allclose(out["range_exp"], r0 * alpha, atol=1e-10)
    np.testing.assert_allclose(out["alpha"], alpha, atol=1e-12)
    np.testing.assert_allclose(out["range_med"], np.where(alpha > 0.5, r0, 0.0), atol=1e-12)


def test_lidar_median_is_first_crossing_and_expected_range_blends():
    lid = small_lidar()
    near = one_gaussian((6.0, 0.0, 0.0), (0.3, 0.3, 0.3), opacity=0.45, feature=(1.0,))
    mid = one_gaussian((9.0, 0.0, 0.0), (0.3, 0.45, 0.45), opacity=0.8, feature=(1.0,))
    far = one_gaussian((12.0, 0.0, 0.0), (0.3, 0.6, 0.6), opacity=0.7, feature=(1.0,))
    out = oracle.render(stack(far, near, mid), lid)  # input order must not matter
    k = 7 * 256 + 0       # beam 7 (-1 deg), azimuth bin 0
    a1 = oracle.render(near, lid)["alpha"][k]
    a2 = oracle.render(mid, lid)["alpha"][k]
    a3 = oracle.render(far, lid)["alpha"][k]
    # transmittance drops below one half at the middle Gaussian and stays below after it
    assert 0 < a1 < 0.5 and (1 - a1) * (1 - a2) < 0.5 and a3 > 0.05
    assert out["range_med"][k] == pytest.approx(9.0, rel=1e-12)
    T = [1.0, 1 - a1, (1 - a1) * (1 - a2)]
    assert out["range_exp"][k] == pytest.approx(6.0 * a1 * T[0] + 9.0 * a2 * T[1] + 12.0 * a3 * T[2], rel=1e-12)
    assert out["T"][k] == pytest.approx(T[2] * (1 - a3), rel=1e-12)


def test_rolling_shutter_shifts_mean_by_row_time():
    vs = np.array([3.0, 0.0, 0.0])  # sensor moving right: static points drift left in the image
    cam = front_camera(width=64, height=64, f=60.0, lin_vel=vs, rs_time=0.05)
    g = one_gaussian((5.0, 0.0, 0.0), (0.2, 0.15, 0.15), opacity=0.9)
    p = oracle.project(g, cam)
    rec = p["rec"][0]
    assert rec[7] == pytest.approx(-60 * 3.0 / 5.0, rel=1e-6)
    r = oracle.render(g, cam)
    a = r["F"][:, 0].reshape(64, 64)
    cols = np.arange(64) + 0.5
    for row in (8, 32, 55):
        t = ((row + 0.5) / 64 - 0.5) * 0.05
        w = a[row]
        if w.sum() < 1e-6:
            continue
        centre = (w * cols).sum() / w.sum()
        assert centre == pytest.approx(rec[0] + rec[7] * t, abs=0.05)


# ----------------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------------

def test_empty_scene():
    for s in (front_camera(), small_lidar()):
        r = oracle.render(empty_scene(), s)
        assert np.all(r["F"] == 0) and np.all(r["T"] == 1)
        if s.kind == "lidar":
            assert np.all(r["range_exp"] == 0) and np.all(r["range_med"] == 0)


def test_constant_features_give_c_times_opacity():
    g, sensors = scenes.tiny_frame()
    g = dict(g)
    g["features"] = np.full_like(g["features"], 0.37)
    for s in sensors:
        r = oracle.render(g, s)
        np.testing.assert_allclose(r["F"], 0.37 * (1 - r["T"])[:, None] * np.ones((1, 3)), atol=1e-12)
        assert (r["T"] < 0.99).mean() > 0.05


def test_zero_motion_rolling_shutter_equals_global_shutter():
    g, sensors = scenes.tiny_frame()
    cam = sensors[0]
    cam_rs = front_camera(rs_time=0.03)
    a, b = oracle.render(g, cam), oracle.render(g, cam_rs)
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["T"], b["T"])
    lid_rs = small_lidar(sweep_time=0.1)
    a, b = oracle.render(g, sensors[1]), oracle.render(g, lid_rs)
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["range_exp"], b["range_exp"])


def test_lidar_rotation_by_one_tile_shifts_columns():
    g, sensors = scenes.tiny_frame()
    lid = sensors[1]
    ang = 32 * float(np.float32(lid.az_res))
    Rz = rodrigues([0, 0, ang])
    qz = np.array([math.cos(ang / 2), 0, 0, math.sin(ang / 2)])
    g64 = {k: np.asarray(v, np.float64) for k, v in g.items()}
    rot = dict(g64)
    rot["means"] = g64["means"] @ Rz.T
    rot["quats"] = np.stack([quat_mul(qz, q) for q in g64["quats"]])
    a, b = oracle.render(g64, lid), oracle.render(rot, lid)
    Fa = a["F"].reshape(16, 256, 3)
    Fb = b["F"].reshape(16, 256, 3)
    ok = ~(a["marginal"].reshape(16, 256) | np.roll(b["marginal"].reshape(16, 256), -32, axis=1))
    # 256 x FP32(res) is not exactly 2 pi, so Gaussians crossing the seam move by ~1e-7 rad
    # relative to the rays of the wrapped column; elsewhere the shift is exact.
    seam = np.zeros((16, 256), bool)
    seam[:, 224:] = True
    seam[:, :32] = True
    Fr = np.roll(Fb, -32, axis=1)
    np.testing.assert_allclose(Fr[ok & ~seam], Fa[ok & ~seam], atol=1e-9)
    np.testing.assert_allclose(Fr[ok & seam], Fa[ok & seam], atol=1e-5)
    assert ok.mean() > 0.98 and np.abs(Fa[seam]).max() > 0.1


def test_permuting_gaussians_keeps_render():
    g, sensors = scenes.tiny_frame()
    perm = np.random.default_rng(3).permutation(len(g["opacities"]))
    gp = {k: v[perm] for k, v in g.items()}
    for s in sensors:
        a, b = oracle.render(g, s), oracle.render(gp, s)
        ok = ~(a["marginal"] | b["marginal"])
        np.testing.assert_allclose(a["F"][ok], b["F"][ok], atol=1e-12)


# ----------------------------------------------------------------------------------
# Tiling against brute force
# ----------------------------------------------------------------------------------

def test_camera_tile_rects_match_brute_force():
    g, sensors = scenes.tiny_frame()
    cam = sensors[0]
    p = oracle.project(g, cam)
    ntx, nty = 8, 6
    tx = np.arange(ntx)
    ty = np.arange(nty)
    for i in np.where(p["visible"])[0]:
        rec = p["rec"][i]
        xs = ((tx + 1) * 16 > rec[0] - rec[14]) & (tx * 16 < rec[0] + rec[14])
        ys = ((ty + 1) * 16 > rec[1] - rec[15]) & (ty * 16 < rec[1] + rec[15])
        x0, y0, x1, y1 = p["rect"][i]
        assert np.array_equal(np.where(xs)[0], np.arange(x0, x1)), i
        assert np.array_equal(np.where(ys)[0], np.arange(y0, y1)), i


def _lidar_columns_brute(lo, hi, W, M):
    """Columns whose ray azimuths [kW, min((k+1)W, 2pi)) meet [lo, hi] on the circle."""
    out = []
    for k in range(M):
        a, b = k * W, min((k + 1) * W, 2 * math.pi)
        if any(max(a, lo + s) < min(b, hi + s) for s in (-2 * math.pi, 0.0, 2 * math.pi)):
            out.append(k)
    return out


@pytest.mark.parametrize("n_az, sweep", [(256, 0.0), (1080, 0.1), (2000, 0.05)])
def test_lidar_tiles_match_brute_force(n_az, sweep):
    g = scenes.driving_gaussians(3000, 77, channels=2, min_radius=1.0)
    vs, ws = np.array([10.0, 0, 0]), np.array([0, 0, 0.2])
    elev = scenes.nonuniform_elevations(32)
    lid = scenes.Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=n_az, az_res=2 * math.pi / n_az,
                       sweep_time=sweep, eps2d=1e-6, lin_vel=vs, ang_vel=ws)
    p = oracle.project(g, lid)
    W = 32 * float(np.float32(lid.az_res))
    M = -(-n_az // 32)
    el = np.asarray(elev, np.float32).astype(np.float64)
    bnd = np.concatenate([[el[0] - (el[1] - el[0]) / 2], (el[7:-1:8] + el[8::8]) / 2,
                          [el[-1] + (el[-1] - el[-2]) / 2]])
    wrapped = 0
    for i in np.where(p["visible"] & ~p["marginal"])[0]:
        rec = p["rec"][i]
        lo, hi = rec[0] - rec[14], rec[0] + rec[14]
        cols = _lidar_columns_brute(lo, hi, W, M)
        x0, y0, x1, y1 = p["rect"][i]
        got = sorted({k % M for k in range(x0, x1)})
        assert got == cols, (i, lo, hi, x0, x1)
        assert x1 - x0 == len(got)
        rows = [j for j in range(4) if bnd[j] < rec[1] + rec[15] and bnd[j + 1] > rec[1] - rec[15]]
        assert list(range(y0, y1)) == rows
        wrapped += (x0 < 0) or (x1 > M)
    assert wrapped > 0


def test_isect_list_is_sorted_by_tile_depth_id():
    g, sensors = scenes.tiny_frame()
    for s in sensors:
        p = oracle.project(g, s)
        tiles, ids = oracle.isect_list(g, s, p)
        M = -(-s.width // 16) if s.kind == "camera" else -(-s.n_az // 32)
        ref = []
        for i in np.where(p["n_tiles"] > 0)[0]:
            x0, y0, x1, y1 = p["rect"][i]
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    ref.append((ty * M + tx % M, p["rec"][i, 6], i))
        ref.sort()
        assert np.array_equal(tiles, [r[0] for r in ref]) and np.array_equal(ids, [r[2] for r in ref])


# ----------------------------------------------------------------------------------
# Gradients: analytic reverse mode vs central finite differences of the forward
# ----------------------------------------------------------------------------------

def _loss(g, s, w, los_range=None):
    r = oracle.render(g, s, guard=0.0, los_range=los_range)
    L = (w["F"] * r["F"]).sum() + (w["T"] * r["T"]).sum()
    if s.kind == "lidar":
        L += (w["D"] * r["range_exp"]).sum() + (w["A"] * r["alpha"]).sum()
    if los_range is not None:
        L += (w["L"] * r["los"]).sum()
    return L, r["count"]


def _weights(s, C, seed):
    rng = np.random.default_rng(seed)
    n = s.n_rays
    return {"F": rng.normal(size=(n, C)), "T": rng.normal(size=n), "D": rng.normal(size=n) * 0.1,
            "A": rng.normal(size=n), "L": rng.normal(size=n)}


def _fd_check(g, s, seed, h=1e-6, los_range=None):
    C = g["features"].shape[1]
    w = _weights(s, C, seed)
    an = oracle.render_backward(g, s, w["F"], w["T"], w["D"] if s.kind == "lidar" else None,
                                w["A"] if s.kind == "lidar" else None, gL=w["L"], los_range=los_range)
    _, c0 = _loss(g, s, w, los_range)
    checked = 0
    for key in ("means", "scales", "quats", "opacities", "velocities", "features"):
        arr = g[key]
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            gp = {k: v.copy() for k, v in g.items()}
            gm = {k: v.copy() for k, v in g.items()}
            step = h * max(1.0, abs(arr[idx]))
            gp[key][idx] += step
            gm[key][idx] -= step
            Lp, cp = _loss(gp, s, w, los_range)
            Lm, cm = _loss(gm, s, w, los_range)
            assert np.array_equal(cp, c0) and np.array_equal(cm, c0), f"discontinuity at {key}{idx}"
            num[idx] = (Lp - Lm) / (2 * step)
        scale = max(np.abs(num).max(), 1e-8)
        np.testing.assert_allclose(an[key], num, atol=2e-5 * scale, rtol=1e-4, err_msg=key)
        checked += np.count_nonzero(num)
    return checked


def test_camera_gradients_match_finite_differences():
    vs, ws = np.array([0.8, -0.3, 5.0]), np.array([0.03, -0.05, 0.02])
    cam = scenes.Camera(R=scenes.camera_rotation(0.1), t=np.array([0.0, 0.1, 0.0]), width=40, height=30, fx=30,
                        fy=28, cx=20.3, cy=14.8, lin_vel=vs, ang_vel=ws, rs_time=0.04, time_offset=0.003,
                        tile_w=8, tile_h=8)
    g = random_small_scene(21, 7, (3.0, -2.0, -1.5), (7.0, 2.0, 1.5), channels=3)
    # one Gaussian far off to the side exercises the clamped part of the Jacobian
    g["means"][6] = (3.5, -4.2, 0.3)
    g["scales"][6] = (0.6, 0.9, 0.5)
    assert _fd_check(g, cam, seed=1) > 40


def test_lidar_gradients_match_finite_differences():
    vs, ws = np.array([12.0, 0.5, 0.0]), np.array([0.0, 0.02, 0.1])
    lid = small_lidar(n_beams=8, n_az=96, lo=-12, hi=10, R=rodrigues([0, 0, 0.2]), lin_vel=vs, ang_vel=ws,
                      sweep_time=0.1, eps2d=2e-5, tile_el=4, tile_az=16)
    g = random_small_scene(33, 6, (-6.0, -6.0, -1.0), (6.0, 6.0, 1.0), channels=2, log_scale=(-1.2, 0.3))
    g["means"][0] = (5.0, -0.05, 0.0)     # straddles the azimuth wrap
    assert _fd_check(g, lid, seed=2) > 40


def _fd_sensor_check(g, s, seed, h=1e-5):
    """Gradients with respect to the sensor's linear and angular velocity (and a camera's
    time offset), translation and rotation against central differences of the rendered
    loss.  Rays whose blended set changes under any of the perturbations (a discrete
    alpha or tile decision within the step) get zero weight."""
    import dataclasses
    C = g["features"].shape[1]
    w = _weights(s, C, seed)
    c0 = oracle.render(g, s, guard=0.0)["count"]
    # every perturbed sensor, as (label, sensor at +, sensor at -, applied parameter change)
    R0 = np.asarray(s.R, np.float64)
    R0f = R0.astype(np.float32).astype(np.float64)

    def applied_rot(Rm):   # rotation a rounded FP32 matrix applies to the rounded base
        A = Rm.astype(np.float32).astype(np.float64) @ R0f.T
        return 0.5 * np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])

    cases = []
    fields = [("lin_vel", k) for k in range(3)] + [("ang_vel", k) for k in range(3)] + [("t", k) for k in range(3)]
    if s.kind == "camera":
        fields.append(("time_offset", None))
    for name, k in fields:
        base = getattr(s, name)
        x0 = float(base if k is None else base[k])
        step = h * max(1.0, abs(x0))
        # sensor parameters reach the renderer as FP32: difference by the rounded values
        xp, xm = float(np.float32(x0 + step)), float(np.float32(x0 - step))

        def moved(xv, name=name, k=k, base=base):
            if k is None:
                return dataclasses.replace(s, **{name: xv})
            v = np.array(base, dtype=np.float64).copy()
            v[k] = xv
            return dataclasses.replace(s, **{name: v})

        cases.append(((name, k), moved(xp), moved(xm), xp - xm))
    hr = 1e-4
    for k in range(3):
        e = np.zeros(3)
        e[k] = hr
        Rp, Rm = rodrigues(e) @ R0, rodrigues(-e) @ R0
        cases.append((("rot", k), dataclasses.replace(s, R=Rp), dataclasses.replace(s, R=Rm),
                      applied_rot(Rp) - applied_rot(Rm)))
    keep = np.ones(s.n_rays, bool)
    for _, sp, sm_, _ in cases:
        keep &= oracle.render(g, sp, guard=0.0)["count"] == c0
        keep &= oracle.render(g, sm_, guard=0.0)["count"] == c0
    assert keep.mean() > 0.98
    w = {k: (v * (keep[:, None] if v.ndim == 2 else keep)) for k, v in w.items()}
    an = oracle.render_backward(g, s, w["F"], w["T"], w["D"] if s.kind == "lidar" else None,
                                w["A"] if s.kind == "lidar" else None)["sensor"]
    checked = 0
    for (name, k), sp, sm_, d in cases:
        Lp, _ = _loss(g, sp, w)
        Lm, _ = _loss(g, sm_, w)
        if name == "rot":
            pred = float(np.dot(an["rot"], d))
            assert Lp - Lm == pytest.approx(pred, rel=1e-3, abs=1e-10), ("rot", k, Lp - Lm, pred)
            checked += (Lp - Lm) != 0
            continue
        num = (Lp - Lm) / d
        got = an[name] if k is None else an[name][k]
        assert got == pytest.approx(num, rel=1e-4, abs=2e-5 * max(1.0, abs(num))), (name, k, got, num)
        checked += num != 0
    return checked


def test_camera_sensor_velocity_and_time_offset_gradients_match_fd():
    """The paper optimises the sensors' linear and angular velocities and the cameras'
    time offset (App. B learning rates, ablation e): their gradients through the pixel
    velocity (Eq. pixel velocity) and the pixel times (Eq. t_pix)."""
    vs, ws = np.array([0.8, -0.3, 5.0]), np.array([0.03, -0.05, 0.02])
    cam = scenes.Camera(R=scenes.camera_rotation(0.1), t=np.array([0.0, 0.1, 0.0]), width=40, height=30, fx=30,
                        fy=28, cx=20.3, cy=14.8, lin_vel=vs, ang_vel=ws, rs_time=0.04, time_offset=0.003,
                        tile_w=8, tile_h=8)
    g = random_small_scene(21, 7, (3.0, -2.0, -1.5), (7.0, 2.0, 1.5), channels=3)
    g["velocities"] = np.random.default_rng(4).normal(0, 1.0, size=(7, 3)).astype(np.float32)
    assert _fd_sensor_check(g, cam, seed=5) == 13


def test_lidar_sensor_velocity_gradients_match_fd():
    vs, ws = np.array([12.0, 0.5, 0.0]), np.array([0.0, 0.02, 0.1])
    lid = small_lidar(n_beams=8, n_az=96, lo=-12, hi=10, R=rodrigues([0, 0, 0.2]), lin_vel=vs, ang_vel=ws,
                      sweep_time=0.1, eps2d=2e-5, tile_el=4, tile_az=16)
    g = random_small_scene(33, 6, (-6.0, -6.0, -1.0), (6.0, 6.0, 1.0), channels=2, log_scale=(-1.2, 0.3))
    assert _fd_sensor_check(g, lid, seed=6) == 12


def test_line_of_sight_gradients_match_finite_differences():
    """App. B line-of-sight term: its gradient (1 on every alpha in front of the return)
    through the alpha chain, against central differences; returns are placed between the
    Gaussians' ranges so that no perturbation moves a Gaussian across the cut."""
    vs, ws = np.array([12.0, 0.5, 0.0]), np.array([0.0, 0.02, 0.1])
    lid = small_lidar(n_beams=8, n_az=96, lo=-12, hi=10, R=rodrigues([0, 0, 0.2]), lin_vel=vs, ang_vel=ws,
                      sweep_time=0.1, eps2d=2e-5, tile_el=4, tile_az=16)
    g = random_small_scene(33, 6, (-6.0, -6.0, -1.0), (6.0, 6.0, 1.0), channels=2, log_scale=(-1.2, 0.3))
    g["means"][0] = (5.0, -0.05, 0.0)
    # ranges of the Gaussians at the rays' times span at most a few cm around |mean|;
    # cuts halfway between consecutive ranges keep a margin of centimetres
    r = np.sort(np.linalg.norm(g["means"].astype(np.float64), axis=1))
    cuts = np.concatenate([[0.5 * r[0]], 0.5 * (r[1:] + r[:-1]), [r[-1] + 1.0]])
    rng = np.random.default_rng(9)
    los_range = rng.choice(cuts, size=lid.n_rays) + 0.8
    assert _fd_check(g, lid, seed=3, los_range=los_range) > 40


def test_line_of_sight_term_sums_alphas_in_front_of_the_return():
    lid = small_lidar()
    near = one_gaussian((6.0, 0.0, 0.0), (0.3, 0.3, 0.3), opacity=0.45, feature=(1.0,))
    mid = one_gaussian((9.0, 0.0, 0.0), (0.3, 0.45, 0.45), opacity=0.8, feature=(1.0,))
    far = one_gaussian((12.0, 0.0, 0.0), (0.3, 0.6, 0.6), opacity=0.7, feature=(1.0,))
    k = 7 * 256 + 0       # beam 7 (-1 deg), azimuth bin 0
    a = [oracle.render(x, lid)["alpha"][k] for x in (near, mid, far)]
    assert min(a) > 0.05
    both = stack(far, near, mid)
    for rp, want in ((10.5, a[0] + a[1]), (9.5, a[0]), (6.5, 0.0), (0.0, 0.0), (100.0, sum(a))):
        out = oracle.render(both, lid, sel=[k], los_range=[rp])
        assert out["los"][0] == pytest.approx(want, rel=1e-12, abs=1e-15), rp
    # a return 0.8 m behind a Gaussian's range: the cut falls on it and the ray is marginal
    out = oracle.render(both, lid, sel=[k], los_range=[9.0 + 0.8])
    assert out["marginal"][0]


# ----------------------------------------------------------------------------------
# Readings where the paper is silent (3DGS conventions): pinned as chosen
# ----------------------------------------------------------------------------------

def test_alpha_is_clamped_at_0999():
    cam = front_camera(width=32, height=32, f=40.0)
    g = one_gaussian((4.0, 0.0, 0.0), (3.0, 3.0, 3.0), opacity=1.0 - 1e-9)
    r = oracle.render(g, cam)
    k = 16 * 32 + 16
    # pixel (16.5, 16.5) is half a pixel from the mean, so o' G exceeds 0.999 before the clamp
    assert r["T"][k] == pytest.approx(1.0 - 0.999, abs=1e-15)


def test_ray_stops_before_transmittance_drops_below_1e4():
    lid = small_lidar()
    layers = [one_gaussian((4.0 + 0.5 * i, 0.0, 0.0), (0.05, 1.0, 1.0), opacity=0.95, feature=(float(i + 1),))
              for i in range(8)]
    # a faint Gaussian behind the terminating one: blending must have stopped, not skipped
    layers.append(one_gaussian((9.0, 0.0, 0.0), (0.05, 2.0, 2.0), opacity=0.05, feature=(100.0,)))
    out = oracle.render(stack(*layers), lid)
    k = 7 * 256 + 0
    a = [oracle.render(l, lid)["alpha"][k] for l in layers]   # single-Gaussian alphas (closed-form pinned)
    T, F, n = 1.0, 0.0, 0
    for i, ai in enumerate(a):
        if T * (1 - ai) < 1e-4:
            break
        F += (i + 1) * ai * T
        T *= 1 - ai
        n += 1
    assert 1 < n < 8 and out["count"][k] == n and a[-1] < 0.1
    assert out["T"][k] == pytest.approx(T, rel=1e-12) and out["T"][k] >= 1e-4
    assert out["F"][k, 0] == pytest.approx(F, rel=1e-12)


# ----------------------------------------------------------------------------------
# App. A.2: lidar points -> rays (ego-motion removal, spherical coordinates, tiles)
# ----------------------------------------------------------------------------------

def test_points_to_rays_static_sensor_spherical_coordinates():
    lid = small_lidar()
    pts = np.array([[10.0, 0.0, 0.0], [0.0, 5.0, 0.0], [1.0, 1.0, math.sqrt(2.0)], [-3.0, -4.0, 0.0]])
    rays, r, _ = oracle.points_to_rays(pts, np.zeros(4), lid)
    np.testing.assert_allclose(r, [10.0, 5.0, 2.0, 5.0], rtol=1e-7)
    np.testing.assert_allclose(rays[:, 0], [0.0, math.pi / 2, math.pi / 4, math.pi + math.atan2(4.0, 3.0)],
                               atol=1e-7)
    np.testing.assert_allclose(rays[:, 1], [0.0, 0.0, math.pi / 4, 0.0], atol=1e-7)


def test_points_to_rays_undoes_ego_motion_to_first_order():
    """A static world point X of an ego-motion-compensated sweep sits, at its capture time
    t, at exp(-t [omega]x) (X - v t) in the moving sensor's frame (exact kinematics for
    constant sensor-frame velocities, translation taken first).  The removal must agree
    with it to second order in t."""
    v, w = np.array([15.0, 0.4, 0.0]), np.array([0.0, 0.02, 0.3])
    lid = small_lidar(lin_vel=v, ang_vel=w)
    rng = np.random.default_rng(3)
    X = rng.uniform(-20, 20, size=(200, 3))
    X[:, 2] = rng.uniform(-2, 2, size=200)
    errs = []
    for t in (0.004, 0.002, 0.001):
        rays, r, _ = oracle.points_to_rays(X, np.full(200, t), lid)
        q = (rodrigues(-t * w) @ (X - t * v).T).T
        want = np.stack([np.mod(np.arctan2(q[:, 1], q[:, 0]), 2 * math.pi),
                         np.arcsin(q[:, 2] / np.linalg.norm(q, axis=1))], 1)
        d = np.abs(rays[:, :2] - want)
        d[:, 0] = np.minimum(d[:, 0], 2 * math.pi - d[:, 0])
        first = t * np.linalg.norm(v + np.cross(w, X), axis=1) / np.linalg.norm(X, axis=1)
        errs.append(d.max())
        assert d.max() < 0.02 * first.min()                  # far below the first-order shift
        np.testing.assert_allclose(rays[:, 2], t)
    assert errs[0] / errs[2] > 10                              # shrinks like t^2 (x16 for t / 4)


def test_points_to_rays_tiles_match_brute_force():
    lid = small_lidar(n_beams=16, n_az=1000)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(4000, 3))
    d[:, 2] *= 0.25
    rays, _, tile = oracle.points_to_rays(d * 20.0, np.zeros(4000), lid)
    el = np.asarray(lid.beam_elev, np.float32).astype(np.float64)
    bnd = np.concatenate([[el[0] - 0.5 * (el[1] - el[0])], 0.5 * (el[7:-1:8] + el[8::8]),
                          [el[-1] + 0.5 * (el[-1] - el[-2])]])
    wphi = 32 * float(np.float32(lid.az_res))
    mphi = (1000 + 31) // 32
    hits = 0
    for k in range(4000):
        phi, om = rays[k, 0], rays[k, 1]
        want = -1
        for ty in range(len(bnd) - 1):
            for tx in range(mphi):
                if tx * wphi <= phi < (tx + 1) * wphi and bnd[ty] <= om < bnd[ty + 1]:
                    want = ty * mphi + tx
        assert tile[k] == want, (k, phi, om, tile[k], want)
        hits += want >= 0
    assert 1000 < hits < 4000


def test_free_rays_at_grid_positions_render_like_the_grid():
    """Rays given as a free list (App. A.2) at exactly the grid's (phi, omega, t) fall in
    the grid cells' tiles and must render identically."""
    lid = small_lidar(n_az=256, lin_vel=np.array([8.0, 0.0, 0.0]), sweep_time=0.1)
    g = random_small_scene(5, 60, (-12.0, -12.0, -2.0), (12.0, 12.0, 2.0), channels=2, log_scale=(-1.0, 0.4))
    grid = oracle.render(g, lid)
    el = np.asarray(lid.beam_elev, np.float32).astype(np.float64)
    res = float(np.float32(lid.az_res))
    a = np.arange(256)
    phi = np.tile((a + 0.5) * res, len(el))
    om = np.repeat(el, 256)
    t = np.tile(((a + 0.5) / 256 - 0.5) * float(np.float32(lid.sweep_time)), len(el))
    free = oracle.render(g, lid, free_rays=np.stack([phi, om, t], 1))
    assert grid["count"].sum() > 500
    np.testing.assert_array_equal(free["count"], grid["count"])
    # free rays reach the renderer as FP32 (phi within 2.4e-7 of the grid's FP64 value)
    np.testing.assert_allclose(free["F"], grid["F"], atol=1e-5)
    np.testing.assert_allclose(free["range_exp"], grid["range_exp"], atol=1e-4)


def test_cap_rays_keeps_the_lowest_priorities_and_samples_uniformly():
    """Training-time cap of App. A.2: tiles at or under the cap keep every ray; over-full
    tiles keep exactly cap rays; with priorities equal to the ray index the first cap
    rays survive; under uniform random priorities every ray of a tile survives with
    probability cap / count (a uniform shuffle)."""
    tile = np.array([0] * 10 + [1] * 3 + [-1] * 2 + [2] * 6)
    keep, lists = oracle.cap_rays(tile, np.arange(len(tile)), 4)
    assert keep[10:13].all() and not keep[13:15].any()
    np.testing.assert_array_equal(np.nonzero(keep[:10])[0], [0, 1, 2, 3])
    np.testing.assert_array_equal(lists[2], [15, 16, 17, 18])
    prio = np.array([5, 5, 1, 9, 0, 7, 7, 3, 2, 8] + [0] * 11)
    keep, lists = oracle.cap_rays(tile, prio, 4)
    np.testing.assert_array_equal(lists[0], [4, 2, 8, 7])              # ties broken by index below
    keep, lists = oracle.cap_rays(tile, np.r_[np.full(10, 3), np.zeros(11)], 4)
    np.testing.assert_array_equal(lists[0], [0, 1, 2, 3])
    rng = np.random.default_rng(9)
    big = np.repeat([0, 1], [300, 200])
    hits = np.zeros(500)
    for _ in range(400):
        k, _ = oracle.cap_rays(big, rng.integers(0, 2**32, size=500, dtype=np.uint64), 256)
        assert k[:300].sum() == 256 and k[300:].all()
        hits += k
    frac = hits[:300] / 400
    assert abs(frac.mean() - 256 / 300) < 1e-12 and frac.min() > 0.7 and frac.max() < 0.97


# ----------------------------------------------------------------------------------
# Opacity-aware tile extent (the alternative to the 3-sigma box)
# ----------------------------------------------------------------------------------

def _support_scene():
    """Rolling-shutter camera and spinning lidar, moving sensors and moving Gaussians of
    high and low opacity (high opacity is where the 3-sigma box cuts the footprint)."""
    import dataclasses
    g = random_small_scene(31, 120, (4.0, -6.0, -3.0), (16.0, 6.0, 3.0), channels=3, log_scale=(-1.2, 0.4))
    g["opacities"] = np.where(np.arange(120) % 2 == 0, 0.97, g["opacities"])
    cam = front_camera(rs_time=0.03, time_offset=0.003, lin_vel=np.array([0.3, 0.0, 10.0]),
                       ang_vel=np.array([0.0, 0.04, 0.0]))
    lid = small_lidar(sweep_time=0.1, lin_vel=np.array([10.0, 0.2, 0.0]), ang_vel=np.array([0.0, 0.0, 0.1]))
    return g, cam, lid, dataclasses.replace


def test_opacity_aware_extent_makes_the_tile_predicate_redundant():
    """With the opacity-aware box the tiles hold every Gaussian that reaches alpha >= 1/255
    anywhere in them at any ray time, so rendering through the tile lists equals the
    per-pixel definition over every visible Gaussian, exactly -- while the paper's 3-sigma
    box drops parts of the high-opacity footprints (alpha at 3 sigma is 0.011 o')."""
    g, cam, lid, replace = _support_scene()
    for s in (cam, lid):
        sa = replace(s, support=1)
        tiled = oracle.render(g, sa)
        full = oracle.render(g, sa, every_gaussian=True)
        assert tiled["count"].sum() > 2000
        np.testing.assert_array_equal(tiled["F"], full["F"])
        np.testing.assert_array_equal(tiled["T"], full["T"])
        np.testing.assert_array_equal(tiled["count"], full["count"])
        if s.kind == "lidar":
            np.testing.assert_array_equal(tiled["range_exp"], full["range_exp"])
    # the 3-sigma box: the camera's 16-px tiles cut high-opacity footprints (the lidar's
    # wide tiles happen to contain them here)
    cut = oracle.render(g, cam)
    cut_full = oracle.render(g, cam, every_gaussian=True)
    d = np.abs(cut["F"] - cut_full["F"]).max()
    assert 1e-3 < d < 0.2, d


def test_opacity_aware_box_is_the_bounding_box_of_the_alpha_ellipse():
    """Static Gaussians, camera: the tile rectangle equals the tiles spanned by the ellipse
    {alpha >= 1/255} traced point by point (the boundary d = m + k L u(theta), with L a
    Cholesky factor of Sigma' and k^2 = 2 ln(255 o')), wherever no traced edge lies within
    0.01 px of a tile boundary."""
    import dataclasses
    g = random_small_scene(32, 200, (4.0, -5.0, -3.0), (14.0, 5.0, 3.0), channels=1, log_scale=(-1.5, 0.5),
                           dynamic=False)
    cam = dataclasses.replace(front_camera(), support=1)
    p = oracle.project(g, cam)
    th = np.linspace(0.0, 2.0 * np.pi, 20001)
    checked = 0
    for i in np.nonzero(p["visible"])[0]:
        r = p["rec"][i]
        Sig = np.array([[r[10], r[11]], [r[11], r[12]]])
        Lc = np.linalg.cholesky(Sig)
        k = math.sqrt(2.0 * math.log(255.0 * r[5]))
        pts = r[:2, None] + k * (Lc @ np.stack([np.cos(th), np.sin(th)]))
        lo, hi = pts.min(axis=1), pts.max(axis=1)
        edges = np.array([lo[0], hi[0], lo[1], hi[1]]) / 16.0
        if np.any(np.abs(edges - np.round(edges)) < 0.01 / 16):
            continue
        ntx, nty = -(-cam.width // 16), -(-cam.height // 16)
        want = [min(max(math.floor(lo[0] / 16), 0), ntx), min(max(math.floor(lo[1] / 16), 0), nty),
                min(max(math.ceil(hi[0] / 16), 0), ntx), min(max(math.ceil(hi[1] / 16), 0), nty)]
        np.testing.assert_array_equal(p["rect"][i], want)
        checked += 1
    assert checked > 100


def test_sweep_time_margins_cover_every_grid_ray_that_can_blend():
    """Lidar box option 2: a grid ray at azimuth phi fires at t(phi) = c phi - t_sweep/2, so
    the margins only need the motion at those times.  Brute force over every azimuth bin:
    each bin whose ray sees the moving mean within the spatial extent lies inside the
    tightened azimuth box, and the mean's elevation at those rays' times lies inside the
    tightened elevation box -- and the boxes are smaller than the symmetric ones."""
    import dataclasses
    g, cam, lid, replace = _support_scene()
    lid = replace(lid, support=2)
    p = oracle.project(g, lid)
    rec = p["rec"]
    half = 0.5 * float(np.float32(lid.sweep_time))
    res = float(np.float32(lid.az_res))
    a = np.arange(lid.n_az)
    phi_a = (a + 0.5) * res
    t_a = ((a + 0.5) / lid.n_az - 0.5) * float(np.float32(lid.sweep_time))
    tightened = checked = 0
    for i in np.nonzero(p["visible"])[0]:
        r = rec[i]
        phi, om, va, vb = r[0], r[1], r[7], r[8]
        es, eo = r[14] - abs(va) * half, r[15] - abs(vb) * half
        if not (phi - r[14] >= 0 and phi + r[14] < 2 * np.pi):
            continue   # the seam keeps the symmetric box
        hit = np.abs(phi_a - (phi + va * t_a)) <= es
        if not hit.any():
            continue
        checked += 1
        assert (phi_a[hit] >= phi - r[16] - 1e-12).all() and (phi_a[hit] <= phi + r[17] + 1e-12).all()
        om_t = om + vb * t_a[hit]
        assert (om_t - eo >= om - r[18] - 1e-12).all() and (om_t + eo <= om + r[19] + 1e-12).all()
        assert r[16] <= r[14] + 1e-12 and r[17] <= r[14] + 1e-12
        tightened += (r[16] + r[17] < 2 * r[14] - 1e-9)
    assert checked > 50 and tightened > checked // 2


def test_sweep_time_margins_keep_the_per_ray_definition():
    """With both options (opacity-aware extent, sweep-time margins) the lidar's tile lists
    still hold every Gaussian a grid ray can blend: rendering through them equals the
    per-ray definition over every visible Gaussian exactly, with fewer intersections."""
    g, cam, lid, replace = _support_scene()
    both, aware = replace(lid, support=3), replace(lid, support=1)
    tiled = oracle.render(g, both)
    full = oracle.render(g, both, every_gaussian=True)
    np.testing.assert_array_equal(tiled["F"], full["F"])
    np.testing.assert_array_equal(tiled["range_exp"], full["range_exp"])
    np.testing.assert_array_equal(tiled["count"], full["count"])
    assert tiled["count"].sum() > 1000
    assert len(oracle.isect_list(g, both)[0]) < len(oracle.isect_list(g, aware)[0])
