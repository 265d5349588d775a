"""FP64 CPU oracle for the SplatAD camera/lidar rasterizer (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never does.

The numerical work lives in ``splat_oracle.c`` (plain C, FP64, OpenMP over
rays); this module only builds it with gcc and marshals numpy arrays through
ctypes.  Functions and the paper passages they follow:

* :func:`project`        -- Sec. 3.2 projection / AABB / tiles; Sec. 3.3 and
                            App. A.1 for the lidar (spherical projection, J^S,
                            azimuth wrap, elevation loop).
* :func:`isect_list`     -- Sec. 3.2 / 3.3 tile duplication and depth (range)
                            sort: pairs ordered by (tile, depth, id).
* :func:`render`         -- Eq. (t_pix), (alpha blend), (alpha), (delta);
                            Sec. 3.3 expected range (r + v_r t) and median range.
* :func:`render_backward`-- reverse mode of the above, then the projection
                            chain rule back to means, scales, quaternions,
                            opacities, velocities and features.
* :mod:`oracle.head`     -- the per-ray MLP decoder (Sec. 3.3, App. B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

GUARD_PX = 1e-4     # camera tile-edge guard band, pixels
GUARD_RAD = 2e-6    # lidar tile-edge guard band, radians
GUARD_RAD_SWEEP = 2e-5   # the same with the sweep-time margins


def build(force: bool = False) -> str:
    """Compile ``splat_oracle.c`` (and the head oracle) into ``liboracle.so``."""
    srcs = [os.path.join(_HERE, "splat_oracle.c"), os.path.join(_HERE, "head_oracle.c")]
    srcs = [s for s in srcs if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _declare(L):
    L.oracle_project.restype = ctypes.c_int
    L.oracle_project.argtypes = [_I64] + [_P] * 7 + [ctypes.c_double] + [_P] * 7
    L.oracle_isect_list.restype = _I64
    L.oracle_isect_list.argtypes = [_I64, _P, _P, _P, _P, _I64, _P, _P]
    L.oracle_render.restype = ctypes.c_int
    L.oracle_render.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int] + [_P] * 3 + [_I64, ctypes.c_double, _I64] +
                                [_P] * 8 + [ctypes.c_double, _P])
    L.oracle_tile_margin.restype = ctypes.c_int
    L.oracle_tile_margin.argtypes = [_P, _P, _I64, _P, _P, _P]
    L.oracle_render_variants.restype = ctypes.c_int
    L.oracle_render_variants.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int] + [_P] * 3 +
                                         [_I64, ctypes.c_double, _I64, _P, _P, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int] + [_P] * 8)
    L.oracle_render_backward.restype = ctypes.c_int
    L.oracle_render_backward.argtypes = ([_I64] + [_P] * 6 + [ctypes.c_int] + [_P] * 3 + [_I64, _I64] + [_P] * 13 +
                                         [ctypes.c_double, _P, _P])
    L.oracle_projection_backward.restype = ctypes.c_int
    L.oracle_projection_backward.argtypes = [_I64] + [_P] * 14
    L.oracle_jacobian.restype = ctypes.c_int
    L.oracle_jacobian.argtypes = [_P, _P, _P, ctypes.c_double, _P, _P, _P, _P, _P]
    if hasattr(L, "head_forward"):
        from . import head as _head
        _head._declare(L)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    """Input array as FP64.  FP32 arrays (what the library receives) are promoted
    exactly; FP64 arrays pass unchanged, so finite-difference tests can perturb
    parameters far below FP32 resolution."""
    if a is None:
        return None
    a = np.asarray(a)
    if a.dtype != np.float64:
        a = a.astype(np.float32)
    return np.ascontiguousarray(a, dtype=np.float64)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _r32(x) -> float:
    """Round a parameter through FP32, exactly as the library receives it."""
    return float(np.float32(x))


def sensor_params(s) -> np.ndarray:
    """Flat FP64 parameter vector of a sensor (values rounded through FP32)."""
    P = np.zeros(40, dtype=np.float64)
    P[1:10] = np.asarray(s.R, dtype=np.float32).reshape(9)
    P[10:13] = np.asarray(s.t, dtype=np.float32)
    P[13:16] = np.asarray(s.lin_vel, dtype=np.float32)
    P[16:19] = np.asarray(s.ang_vel, dtype=np.float32)
    if s.kind == "camera":
        P[0] = 0
        P[19:31] = [s.width, s.height, _r32(s.fx), _r32(s.fy), _r32(s.cx), _r32(s.cy), _r32(s.rs_time),
                    _r32(s.time_offset), _r32(s.eps2d), _r32(s.near), s.tile_w, s.tile_h]
    else:
        P[0] = 1
        P[19:27] = [s.n_beams, s.n_az, _r32(s.az_res), _r32(s.sweep_time), _r32(s.eps2d), _r32(s.r_min),
                    s.tile_az, s.tile_el]
    P[31] = getattr(s, "support", 0)   # tile extent flags: 1 opacity-aware, 2 lidar sweep-time margins
    return P


def _sensor_array(a):
    """Sensor-side arrays always reach the renderer in FP32; round them the same way."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32), dtype=np.float64)


def _elev(s):
    return _sensor_array(s.beam_elev) if s.kind == "lidar" else None


def _rays(s):
    return _sensor_array(s.rays.reshape(-1, 3)) if (s.kind == "lidar" and s.rays is not None) else None


def _g(g):
    return [_f32(g["means"]), _f32(g["scales"]), _f32(g["quats"]), _f32(g["opacities"]), _f32(g.get("velocities"))]


def guard_for(s) -> float:
    if s.kind == "camera":
        return GUARD_PX
    # the sweep-time margins go through a division and more FP32 steps on the GPU
    return GUARD_RAD_SWEEP if (getattr(s, "support", 0) & 2) else GUARD_RAD


def n_tiles_of(s):
    if s.kind == "camera":
        return (-(-s.width // s.tile_w)) * (-(-s.height // s.tile_h))
    return (-(-s.n_az // s.tile_az)) * (s.n_beams // s.tile_el)


def project(g: dict, s, guard: float | None = None) -> dict:
    """Per-Gaussian projection of one sensor (FP64).

    Returns rec (n,20): [mean_a, mean_b, conic a, b, c, o', depth, v_a, v_b, v_r,
    Sigma'_aa, Sigma'_ab, Sigma'_bb, compensation, extent_a, extent_b, lidar box below / above the mean
    along a and b], rect (n,4),
    outer and inner rects of marginal Gaussians (tiles whose membership FP32 rounding
    could change lie between the two), n_tiles, visible and marginal flags.
    """
    L = lib()
    n = len(g["opacities"])
    m = _g(g)
    P = sensor_params(s)
    guard = guard_for(s) if guard is None else guard
    rec = np.zeros((n, 20)); rect = np.zeros((n, 4), np.int32); orect = np.zeros((n, 4), np.int32)
    irect = np.zeros((n, 4), np.int32)
    nt = np.zeros(n, np.int32); vis = np.zeros(n, np.uint8); marg = np.zeros(n, np.uint8)
    el = _elev(s)
    L.oracle_project(n, *[_ptr(a) for a in m], _ptr(P), _ptr(el), guard, _ptr(rec), _ptr(rect), _ptr(orect),
                     _ptr(irect), _ptr(nt), _ptr(vis), _ptr(marg))
    return {"rec": rec, "rect": rect, "orect": orect, "irect": irect, "n_tiles": nt, "visible": vis.astype(bool),
            "marginal": marg.astype(bool)}


def isect_list(g: dict, s, proj: dict | None = None):
    """Sorted (tile, gaussian id) intersection list of one sensor."""
    L = lib()
    proj = project(g, s) if proj is None else proj
    n = len(g["opacities"])
    P = sensor_params(s)
    total = int(proj["n_tiles"].astype(np.int64).sum())
    tiles = np.zeros(max(total, 1), np.int32); ids = np.zeros(max(total, 1), np.int32)
    got = L.oracle_isect_list(n, _ptr(P), _ptr(proj["rec"]), _ptr(proj["rect"]), _ptr(proj["n_tiles"]), total,
                              _ptr(tiles), _ptr(ids))
    assert got <= total   # fewer with the camera tile cull (support flag 4)
    return tiles[:got], ids[:got]


def tile_margin(g: dict, s, tiles, ids, proj: dict | None = None) -> np.ndarray:
    """Camera tile-cull margins (support flag 4) of (sensor-local tile, Gaussian index)
    pairs: positive where the Gaussian cannot reach alpha >= 1/255 at any pixel of the
    tile (the pair is not listed), by how much of the Mahalanobis form."""
    L = lib()
    proj = project(g, s) if proj is None else proj
    t = np.ascontiguousarray(tiles, dtype=np.int32)
    i = np.ascontiguousarray(ids, dtype=np.int32)
    out = np.zeros(len(t))
    L.oracle_tile_margin(_ptr(sensor_params(s)), _ptr(proj["rec"]), len(t), _ptr(t), _ptr(i), _ptr(out))
    return out


def render(g: dict, s, sel=None, guard: float | None = None, los_range=None, los_eps: float = 0.8,
           free_rays=None, every_gaussian: bool = False) -> dict:
    """Render the selected rays (indices into the sensor's ray grid; None: all).

    Camera ray k is pixel (row, col) = divmod(k, width); lidar ray k is
    (beam, azimuth bin) = divmod(k, n_az).  With los_range (one return range per
    selected lidar ray; <= 0: no return) the line-of-sight term of App. B is returned
    as out["los"]: the summed alpha of the blended Gaussians whose range r_rs lies
    before los_range - los_eps.  With free_rays ((k, 3) phi, omega, t of a lidar, e.g.
    from points_to_rays) those rays are rendered instead of the grid, each in the tile
    its own (phi, omega) falls in (App. A.2).  every_gaussian drops the tile predicate:
    each ray then blends, in depth order, every visible Gaussian that reaches alpha >=
    1/255 at it -- the per-pixel definition without tiles.
    """
    L = lib()
    n = len(g["opacities"])
    m = _g(g)
    feat = _f32(g["features"])
    C = feat.shape[1] if feat.ndim == 2 else 0
    P = sensor_params(s)
    P[32] = 1.0 if every_gaussian else 0.0
    guard = guard_for(s) if guard is None else guard
    sel_arr = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    fr = None if free_rays is None else _sensor_array(np.asarray(free_rays).reshape(-1, 3))
    nfree = 0 if fr is None else len(fr)
    nr = (nfree if fr is not None else s.n_rays) if sel is None else len(sel_arr)
    F = np.zeros((nr, C)); T = np.zeros(nr); De = np.zeros(nr); Dm = np.zeros(nr)
    mg = np.zeros(nr, np.uint8); cnt = np.zeros(nr, np.int32)
    lr = None if los_range is None else _f64(los_range)
    los = np.zeros(nr) if lr is not None else None
    L.oracle_render(n, *[_ptr(a) for a in m], _ptr(feat), C, _ptr(P), _ptr(_elev(s)),
                    _ptr(fr if fr is not None else _rays(s)), nfree, guard, nr, _ptr(sel_arr), _ptr(F), _ptr(T), _ptr(De), _ptr(Dm), _ptr(mg), _ptr(cnt), _ptr(lr),
                    float(los_eps), _ptr(los))
    out = {"F": F, "T": T, "marginal": mg.astype(bool), "marginal_bits": mg, "count": cnt}
    if los is not None:
        out["los"] = los
    if s.kind == "lidar":
        out.update({"range_exp": De, "range_med": Dm, "alpha": 1.0 - T})
    return out


# Kinds of near decisions (bits of the marginal mask), see render_variants.
NEAR_TILE, NEAR_ALPHA_MIN, NEAR_ALPHA_MAX, NEAR_STOP, NEAR_MEDIAN, NEAR_TIE, NEAR_LOS, NEAR_RAY_TILE = (
    1, 2, 4, 8, 16, 32, 64, 128)
MAX_NEAR = 4


def render_variants(g: dict, s, sel=None, guard: float | None = None, los_range=None, los_eps: float = 0.8,
                    free_rays=None, every_gaussian: bool = False, max_dec: int = MAX_NEAR) -> dict:
    """Render the selected rays under every admissible resolution of their near decisions.

    A ray's discrete decisions -- tile membership of a Gaussian whose box edge lies at a
    tile edge, alpha >= 1/255, the stop before T < 1e-4, the T < 1/2 crossing of the
    median range, the order of two blended Gaussians of equal depth, the line-of-sight
    cut -- can go either way in FP32 when the FP64 value lies within the guard band of
    the threshold.  Each way gives a correct render.  Variant 0 is the FP64 render (as
    ``render``); variants 1 .. 2^d - 1 take each non-empty subset of the d near
    decisions the other way, d <= max_dec.  Rays with more near decisions keep variant 0
    only and are reported as unresolved.

    Returns F (rays, V, C), T, range_exp, range_med, los (rays, V), n_var (rays,),
    marginal_bits, n_near, unresolved (n_near > max_dec; rays whose ray tile itself is
    uncertain, free rays only, are unresolved too).  every_gaussian as in ``render``."""
    L = lib()
    n = len(g["opacities"])
    m = _g(g)
    feat = _f32(g["features"])
    C = feat.shape[1] if feat.ndim == 2 else 0
    P = sensor_params(s)
    P[32] = 1.0 if every_gaussian else 0.0
    guard = guard_for(s) if guard is None else guard
    sel_arr = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    fr = None if free_rays is None else _sensor_array(np.asarray(free_rays).reshape(-1, 3))
    nfree = 0 if fr is None else len(fr)
    nr = (nfree if fr is not None else s.n_rays) if sel is None else len(sel_arr)
    V = 1 << max_dec
    F = np.zeros((nr, V, C)); T = np.zeros((nr, V)); De = np.zeros((nr, V)); Dm = np.zeros((nr, V))
    los = np.zeros((nr, V)) if los_range is not None else None
    nvar = np.zeros(nr, np.int32); mg = np.zeros(nr, np.uint8); nd = np.zeros(nr, np.int32)
    lr = None if los_range is None else _f64(los_range)
    rc = L.oracle_render_variants(n, *[_ptr(a) for a in m], _ptr(feat), C, _ptr(P), _ptr(_elev(s)),
                                  _ptr(fr if fr is not None else _rays(s)), nfree, guard, nr, _ptr(sel_arr), _ptr(lr),
                                  float(los_eps), max_dec, V, _ptr(F), _ptr(T), _ptr(De), _ptr(Dm), _ptr(los),
                                  _ptr(nvar), _ptr(mg), _ptr(nd))
    assert rc == 0
    out = {"F": F, "T": T, "n_var": nvar, "marginal_bits": mg, "n_near": nd,
           "unresolved": (nd > max_dec) | ((mg & NEAR_RAY_TILE) != 0)}
    if los is not None:
        out["los"] = los
    if s.kind == "lidar":
        out.update({"range_exp": De, "range_med": Dm, "alpha": 1.0 - T})
    return out


def render_backward(g: dict, s, gF, gT=None, gD=None, gA=None, sel=None, gL=None, los_range=None,
                    los_eps: float = 0.8, free_rays=None) -> dict:
    """Gradients of sum(gF*F) + sum(gT*T) [+ sum(gD*range_exp) + sum(gA*alpha)
    + sum(gL*los)] over the selected rays (None: all rays; the upstream arrays then hold
    one row per selected ray).  out["sensor"] holds the gradients with respect to the
    sensor's linear and angular velocity, (cameras) its time offset, its translation t
    and its rotation (R perturbed as (I + [theta]x) R, theta in the sensor frame)."""
    L = lib()
    n = len(g["opacities"])
    m = _g(g)
    feat = _f32(g["features"])
    C = feat.shape[1]
    P = sensor_params(s)
    out = {"d2": np.zeros((n, 10)), "features": np.zeros((n, C)), "means": np.zeros((n, 3)),
           "scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "opacities": np.zeros(n),
           "velocities": np.zeros((n, 3))}
    ds = np.zeros(16)  # sensor: linear velocity, angular velocity, camera time offset, -, translation, rotation
    sel_arr = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
    fr = None if free_rays is None else _sensor_array(np.asarray(free_rays).reshape(-1, 3))
    L.oracle_render_backward(n, *[_ptr(a) for a in m], _ptr(feat), C, _ptr(P), _ptr(_elev(s)),
                             _ptr(fr if fr is not None else _rays(s)), 0 if fr is None else len(fr),
                             0 if sel_arr is None else len(sel_arr), _ptr(sel_arr),
                             _ptr(_f64(gF)), _ptr(_f64(gT)), _ptr(_f64(gD)), _ptr(_f64(gA)), _ptr(out["d2"]),
                             _ptr(out["features"]), _ptr(out["means"]), _ptr(out["scales"]), _ptr(out["quats"]),
                             _ptr(out["opacities"]), _ptr(out["velocities"]),
                             _ptr(None if los_range is None else _f64(los_range)), float(los_eps), _ptr(_f64(gL)),
                             _ptr(ds))
    out["sensor"] = {"lin_vel": ds[0:3], "ang_vel": ds[3:6], "time_offset": float(ds[6]), "t": ds[8:11],
                     "rot": ds[11:14]}
    return out


def projection_backward(g: dict, s, d2) -> dict:
    L = lib()
    n = len(g["opacities"])
    m = _g(g)
    P = sensor_params(s)
    out = {"means": np.zeros((n, 3)), "scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
           "opacities": np.zeros(n), "velocities": np.zeros((n, 3))}
    L.oracle_projection_backward(n, *[_ptr(a) for a in m], _ptr(P), _ptr(_elev(s)),
                                 _ptr(np.ascontiguousarray(d2, dtype=np.float64)), _ptr(out["means"]),
                                 _ptr(out["scales"]), _ptr(out["quats"]), _ptr(out["opacities"]),
                                 _ptr(out["velocities"]), None)
    return out


def points_to_rays(points, times, s):
    """App. A.2: lidar points (sensor frame at the sweep's reference time, i.e. ego-motion
    compensated) and their capture times -> rays (phi, omega, t), ranges r and tiles.
    The compensation is removed with the sensor's constant velocities (the motion model
    of the rolling-shutter projection): a static point p appears at p - t (v + omega x p)
    in the sensor frame of its capture time.  Each point then takes the tile of a
    zero-extent Gaussian at its (phi, omega): column floor(phi / w_phi) and the row
    whose elevation boundaries contain omega; tile -1 outside the beam fan.  FP64."""
    p = np.asarray(points, np.float32).astype(np.float64).reshape(-1, 3)
    t = np.asarray(times, np.float32).astype(np.float64).reshape(-1)
    v = np.asarray(s.lin_vel, np.float32).astype(np.float64)
    w = np.asarray(s.ang_vel, np.float32).astype(np.float64)
    q = p - t[:, None] * (v[None, :] + np.cross(w[None, :], p))
    r = np.linalg.norm(q, axis=1)
    phi = np.mod(np.arctan2(q[:, 1], q[:, 0]), 2 * np.pi)
    om = np.arcsin(np.clip(q[:, 2] / np.maximum(r, 1e-300), -1.0, 1.0))
    elev = np.asarray(s.beam_elev, np.float32).astype(np.float64)
    nb, tel = len(elev), s.tile_el
    mw = nb // tel
    bnd = [elev[0] - 0.5 * (elev[1] - elev[0])]
    bnd += [0.5 * (elev[k * tel - 1] + elev[k * tel]) for k in range(1, mw)]
    bnd.append(elev[-1] + 0.5 * (elev[-1] - elev[-2]))
    bnd = np.array(bnd)
    mphi = (s.n_az + s.tile_az - 1) // s.tile_az
    wphi = s.tile_az * float(np.float32(s.az_res))
    col = np.minimum(np.floor(phi / wphi).astype(np.int64), mphi - 1)
    row = np.zeros(len(p), np.int64)
    for k in range(1, mw):
        row = np.where(bnd[k] <= om, k, row)
    inside = (om > bnd[0]) & (om < bnd[mw])
    tile = np.where(inside, row * mphi + col, -1)
    return np.stack([phi, om, t], axis=1), r, tile


def cap_rays(tile, priority, cap: int):
    """App. A.2, training: a tile given more rays than it has threads keeps a random
    subset -- the rays are shuffled each iteration and those beyond `cap` dropped.  The
    shuffle is the caller's draw `priority` (one integer per ray): each tile keeps its cap
    rays of smallest (priority, ray index).  Returns the kept mask and, per tile, the kept
    ray indices in that order."""
    tile = np.asarray(tile).reshape(-1)
    pr = np.asarray(priority).astype(np.uint64).reshape(-1)
    keep = np.zeros(len(tile), bool)
    lists = {}
    for t in np.unique(tile[tile >= 0]):
        idx = np.nonzero(tile == t)[0]
        order = sorted(idx.tolist(), key=lambda i: (int(pr[i]), i))[:cap]
        keep[order] = True
        lists[int(t)] = np.array(order, np.int64)
    return keep, lists


def jacobian(mean, scale, quat, opac, s):
    """(visible, J (3x3), sensor-frame covariance, relative velocity w) of one Gaussian."""
    L = lib()
    J = np.zeros(9); Sc = np.zeros(9); w = np.zeros(3)
    vis = L.oracle_jacobian(_ptr(_f32(mean)), _ptr(_f32(scale)), _ptr(_f32(quat)), float(np.float32(opac)),
                            _ptr(sensor_params(s)), _ptr(_elev(s)), _ptr(J), _ptr(Sc), _ptr(w))
    return bool(vis), J.reshape(3, 3), Sc.reshape(3, 3), w


def frame_isect_list(g: dict, sensors) -> tuple[np.ndarray, np.ndarray]:
    """Concatenated list over a frame's sensors with global tile ids (sensor order)."""
    tiles, ids, off = [], [], 0
    for s in sensors:
        t, i = isect_list(g, s)
        tiles.append(t.astype(np.int64) + off)
        ids.append(i)
        off += n_tiles_of(s)
    return np.concatenate(tiles), np.concatenate(ids)
