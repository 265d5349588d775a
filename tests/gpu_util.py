"""Helpers for the GPU parity tests: run a frame through libsplat and compare with
the FP64 oracle on the same seeded inputs.

Discrete decisions that lie within the FP32 guard band of their threshold (a Gaussian's
tile membership, alpha >= 1/255, the stop before T < 1e-4, the T < 1/2 crossing of the
median range, the order of two Gaussians of equal depth, the line-of-sight cut) may go
either way on the GPU.  The oracle renders such a ray once per way of taking them
(``oracle.render_variants``) and a ray passes when the GPU's outputs match one of its
variants within the tolerances below.  Rays with more near decisions than the oracle
enumerates are "unresolved": excluded and counted (none at the sizes tested)."""
import numpy as np
import torch

import oracle
from paper_2411_16816_gb300.render import Frame, gaussians_to_device

DEV = torch.device("cuda:0")

TOL_FEAT = 1e-4     # absolute, rendered features / colour / transmittance / accumulated alpha
TOL_RANGE = 1e-4    # relative (plus 1e-4 m absolute), expected range
TOL_MED = 1e-5      # absolute part of the median-range tolerance (relative part TOL_RANGE)
TOL_GRAD = 1e-3     # relative
CULL_BAND = 5e-3    # camera tile cull: |margin| (units of the Mahalanobis form) of a decision FP32 may flip

# Near decisions that change a ray's gradient by more than FP32 noise when taken the other
# way: membership, alpha >= 1/255, the 0.999 clamp (no gradient through a clamped alpha),
# the order of a depth tie, the line-of-sight cut, an uncertain ray tile.  The stop before
# T < 1e-4 moves only terms of size T (< 1e-4) and the median has no gradient, so rays
# near those two keep their upstream gradient.
GRAD_NEAR = (oracle.NEAR_TILE | oracle.NEAR_ALPHA_MIN | oracle.NEAR_ALPHA_MAX | oracle.NEAR_TIE | oracle.NEAR_LOS |
             oracle.NEAR_RAY_TILE)
CAUSES = {oracle.NEAR_TILE: "tile", oracle.NEAR_ALPHA_MIN: "alpha_min", oracle.NEAR_ALPHA_MAX: "alpha_max",
          oracle.NEAR_STOP: "stop", oracle.NEAR_MEDIAN: "median", oracle.NEAR_TIE: "tie", oracle.NEAR_LOS: "los",
          oracle.NEAR_RAY_TILE: "ray_tile"}


def run(g, sensors, keep_state=True, capacity=None):
    gd = gaussians_to_device(g, DEV)
    fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV, capacity=capacity)
    out = fr.forward(gd, keep_state=keep_state)
    torch.cuda.synchronize()
    return fr, gd, out


def per_sensor(fr, out, key, kind):
    return [v.cpu().numpy().reshape(v.shape[0] * v.shape[1], *v.shape[2:]) for v in fr.split(out[key], kind)]


def variant_errors(kind, got: dict, ref: dict) -> np.ndarray:
    """Normalised error of every (ray, variant): max over the outputs of |GPU - oracle|
    divided by that output's tolerance; a ray matches a variant when it is <= 1.
    got: F (rays, C) and T (camera) or alpha, range_exp, range_med (lidar); optional los."""
    nv = ref["n_var"]
    V = ref["F"].shape[1]
    F = np.asarray(got["F"], np.float64)
    e = np.abs(F[:, None, :] - ref["F"]).max(axis=2, initial=0.0) / TOL_FEAT
    if kind == "camera" and "T" in got:
        e = np.maximum(e, np.abs(np.asarray(got["T"], np.float64)[:, None] - ref["T"]) / TOL_FEAT)
    if kind == "lidar" and "alpha" in got:
        e = np.maximum(e, np.abs(np.asarray(got["alpha"], np.float64)[:, None] - ref["alpha"]) / TOL_FEAT)
    if kind == "lidar" and "range_exp" in got:
        De = np.asarray(got["range_exp"], np.float64)[:, None]
        e = np.maximum(e, np.abs(De - ref["range_exp"]) / (TOL_RANGE + TOL_RANGE * np.abs(ref["range_exp"])))
    if kind == "lidar":
        if "range_med" in got:
            Dm = np.asarray(got["range_med"], np.float64)[:, None]
            e = np.maximum(e, np.abs(Dm - ref["range_med"]) / (TOL_MED + TOL_RANGE * np.abs(ref["range_med"])))
    if "los" in got and "los" in ref:
        e = np.maximum(e, np.abs(np.asarray(got["los"], np.float64)[:, None] - ref["los"]) / TOL_FEAT)
    e[np.arange(V)[None, :] >= nv[:, None]] = np.inf
    return e


def check_variants(kind, got: dict, ref: dict, max_unresolved: float = 0.0, what: str = "") -> dict:
    """Every resolved ray matches one of its oracle variants.  Returns the statistics:
    rays, near (fraction with a near decision), per-cause fractions, the fraction matched
    only by a variant other than the FP64 render, the unresolved fraction and the
    largest normalised error of the best variant."""
    e = variant_errors(kind, got, ref)
    best = e.min(axis=1)
    unres = ref["unresolved"]
    bits = ref["marginal_bits"]
    bad = (best > 1.0) & ~unres
    if bad.any():
        j = np.nonzero(bad)[0][:8]
        detail = [(int(i), float(best[i]), int(bits[i]), int(ref["n_var"][i])) for i in j]
        raise AssertionError(f"{what}: {int(bad.sum())} of {len(best)} rays match no oracle variant "
                             f"(ray, error / tolerance, near bits, variants): {detail}")
    n = max(len(best), 1)
    st = {"rays": len(best), "near": float((bits != 0).mean()) if len(bits) else 0.0,
          "by_cause": {name: float(((bits & b) != 0).mean()) for b, name in CAUSES.items() if ((bits & b) != 0).any()},
          "other_variant": float(((e[:, 0] > 1.0) & ~unres).sum() / n),
          "unresolved": float(unres.mean()) if len(unres) else 0.0,
          "worst": float(best[~unres].max()) if (~unres).any() else 0.0}
    assert st["unresolved"] <= max_unresolved, f"{what}: unresolved fraction {st['unresolved']}"
    return st


def check_render(fr, out, g, sensors, sel=None, max_unresolved=0.0, every_gaussian=False):
    """Compare every sensor's outputs with the oracle's variants (on the selected ray
    indices).  Returns one statistics dict per sensor (see check_variants)."""
    cams = per_sensor(fr, out, "cam_feat", "camera") if fr.cam_idx else []
    camT = per_sensor(fr, out, "cam_T", "camera") if fr.cam_idx else []
    lids = per_sensor(fr, out, "lid_feat", "lidar") if fr.lid_idx else []
    lre = per_sensor(fr, out, "lid_range_exp", "lidar") if fr.lid_idx else []
    lrm = per_sensor(fr, out, "lid_range_med", "lidar") if fr.lid_idx else []
    lal = per_sensor(fr, out, "lid_alpha", "lidar") if fr.lid_idx else []
    ci = li = 0
    stats = []
    for k, s in enumerate(sensors):
        idx = None if sel is None else sel[k]
        ref = oracle.render_variants(g, s, sel=idx, every_gaussian=every_gaussian)
        take = (lambda a: a) if idx is None else (lambda a: a[idx])
        if s.kind == "camera":
            got = {"F": take(cams[ci]), "T": take(camT[ci])}
            ci += 1
        else:
            got = {"F": take(lids[li]), "alpha": take(lal[li]), "range_exp": take(lre[li]),
                   "range_med": take(lrm[li])}
            li += 1
        stats.append(check_variants(s.kind, got, ref, max_unresolved, f"sensor {k} ({s.kind})"))
    print("parity", [(st["rays"], round(st["near"], 5), round(st["other_variant"], 5), st["unresolved"],
                      round(st["worst"], 3), st["by_cause"]) for st in stats])
    return stats


def grad_mask(g, s, sel=None, **kw):
    """1 on the rays whose gradient is decided away from every guard band, else 0."""
    bits = oracle.render(g, s, sel=sel, **kw)["marginal_bits"]
    return ((bits & GRAD_NEAR) == 0).astype(np.float64)


def upstream(fr, sensors, g, seed, with_T=True):
    """Random upstream gradients, zero on the rays with a gradient-relevant near decision."""
    rng = np.random.default_rng(seed)
    C = g["features"].shape[1]
    grads, per = {}, []
    cam_F, cam_T, lid_F, lid_D, lid_A = [], [], [], [], []
    dropped = []
    for s in sensors:
        keep = grad_mask(g, s)
        dropped.append(1 - keep.mean())
        n = s.n_rays
        gF = (rng.normal(size=(n, C)) * keep[:, None]).astype(np.float32)
        gT = (rng.normal(size=n) * keep).astype(np.float32) if with_T else np.zeros(n, np.float32)
        if s.kind == "camera":
            cam_F.append(gF)
            cam_T.append(gT)
            per.append({"gF": gF, "gT": gT})
        else:
            gD = (rng.normal(size=n) * keep * 0.05).astype(np.float32)
            lid_F.append(gF)
            lid_D.append(gD)
            lid_A.append(gT)
            per.append({"gF": gF, "gD": gD, "gA": gT})
    print("gradient rays left out", [round(x, 5) for x in dropped])
    assert max(dropped) < 0.02, dropped
    f32 = lambda xs: torch.as_tensor(np.concatenate(xs).astype(np.float32), device=DEV)
    if cam_F:
        grads["cam_feat"], grads["cam_T"] = f32(cam_F), f32(cam_T)
    if lid_F:
        grads["lid_feat"], grads["lid_range_exp"], grads["lid_alpha"] = f32(lid_F), f32(lid_D), f32(lid_A)
    return grads, per


def sampled_upstream(fr, sensors, g, sel, seed):
    """Upstream gradients on the selected rays of each sensor only (zero elsewhere and on
    rays with a gradient-relevant near decision).  Returns the device dict and, per
    sensor, the selected rays' upstream rows for the oracle (render_backward(sel=))."""
    rng = np.random.default_rng(seed)
    C = g["features"].shape[1]
    cam_F, cam_T, lid_F, lid_D, lid_A, per, dropped = [], [], [], [], [], [], []
    for s, idx in zip(sensors, sel):
        keep = grad_mask(g, s, sel=idx)
        dropped.append(1 - keep.mean())
        n = s.n_rays
        gF, gT = np.zeros((n, C), np.float32), np.zeros(n, np.float32)
        gF[idx] = rng.normal(size=(len(idx), C)) * keep[:, None]
        gT[idx] = rng.normal(size=len(idx)) * keep
        if s.kind == "camera":
            cam_F.append(gF)
            cam_T.append(gT)
            per.append({"gF": gF[idx], "gT": gT[idx], "sel": idx})
        else:
            gD = np.zeros(n, np.float32)
            gD[idx] = rng.normal(size=len(idx)) * keep * 0.05
            lid_F.append(gF)
            lid_D.append(gD)
            lid_A.append(gT)
            per.append({"gF": gF[idx], "gD": gD[idx], "gA": gT[idx], "sel": idx})
    print("gradient rays left out", [round(x, 5) for x in dropped])
    assert max(dropped) < 0.02, dropped
    f32 = lambda xs: torch.as_tensor(np.concatenate(xs), device=DEV)
    grads = {}
    if cam_F:
        grads["cam_feat"], grads["cam_T"] = f32(cam_F), f32(cam_T)
    if lid_F:
        grads["lid_feat"], grads["lid_range_exp"], grads["lid_alpha"] = f32(lid_F), f32(lid_D), f32(lid_A)
    return grads, per


def oracle_grads(g, sensors, per):
    tot = None
    for s, u in zip(sensors, per):
        sel = u.get("sel")
        if s.kind == "camera":
            r = oracle.render_backward(g, s, u["gF"], u["gT"], sel=sel)
        else:
            r = oracle.render_backward(g, s, u["gF"], None, u["gD"], u["gA"], sel=sel)
        sens = r.pop("sensor")
        if tot is None:
            tot = r
            tot["sensor"] = [sens]
        else:
            for k in r:
                tot[k] = tot[k] + r[k]
            tot["sensor"].append(sens)
    return tot


def check_grads(pg, ref, keys=("means", "scales", "quats", "opacities", "features", "velocities"), tol=TOL_GRAD):
    for k in keys:
        if k not in pg or pg[k] is None:
            continue
        got = pg[k].detach().cpu().numpy().astype(np.float64)
        exp = ref[k]
        scale = np.abs(exp).max()
        if scale == 0:
            assert np.abs(got).max() == 0, k
            continue
        rel = np.linalg.norm(got - exp) / np.linalg.norm(exp)
        assert rel <= tol, f"{k}: relative norm error {rel:.2e}"
        np.testing.assert_allclose(got, exp, atol=tol * scale + 1e-6, rtol=0, err_msg=k)


# ----------------------------------------------------------------------------------
# Intersection lists
# ----------------------------------------------------------------------------------

def _rect_has(kind, rects, tiles_x, tx, ty):
    """Vectorised: does rect (x0, y0, x1, y1) hold tile (tx, ty)?  Lidar columns wrap."""
    inside_y = (ty >= rects[:, 1]) & (ty < rects[:, 3])
    if kind == "camera":
        return inside_y & (tx >= rects[:, 0]) & (tx < rects[:, 2])
    d = np.mod(tx - rects[:, 0], tiles_x)
    return inside_y & (d < rects[:, 2] - rects[:, 0])


def compare_lists(fr, g, sensors, which=None):
    """The GPU's intersection lists against the oracle's, sensor by sensor (`which`: the
    sensor indices to compare, default all).  Exact except for:
      * pairs (tile, Gaussian) of a Gaussian whose FP64 box or cull decision lies within
        the guard band, in the tiles between its inner and outer boxes (present or not);
      * the order of two Gaussians whose depths differ by less than 1e-6 (relative): an
        FP32 depth tie, ordered by index on the GPU and by the FP64 depth in the oracle.
    Returns (pairs compared, optional pairs that differ, positions reordered by ties)."""
    tiles, ids = fr.intersections()
    off = 0
    n = len(g["opacities"])
    total = [0, 0, 0]
    for k, s in enumerate(sensors):
        nt = oracle.n_tiles_of(s)
        lo, hi = np.searchsorted(tiles, [off, off + nt])
        if which is not None and k not in which:
            off += nt
            continue
        t_gpu, i_gpu = tiles[lo:hi] - off, ids[lo:hi]
        proj = oracle.project(g, s)
        t_ref, i_ref = oracle.isect_list(g, s, proj)
        t_ref = t_ref.astype(np.int64)
        i_ref = i_ref.astype(np.int64)
        tiles_x = (-(-s.width // s.tile_w)) if s.kind == "camera" else (-(-s.n_az // s.tile_az))
        key_gpu = t_gpu * n + i_gpu
        key_ref = t_ref * n + i_ref
        assert len(np.unique(key_gpu)) == len(key_gpu), f"sensor {k}: duplicate pairs"
        extra = np.setdiff1d(key_gpu, key_ref, assume_unique=True)
        missing = np.setdiff1d(key_ref, key_gpu, assume_unique=True)
        diff = np.concatenate([extra, missing])
        dt, di = diff // n, diff % n
        ok = proj["marginal"][di] & _rect_has(s.kind, proj["orect"][di], tiles_x, dt % tiles_x, dt // tiles_x) & \
            ~_rect_has(s.kind, proj["irect"][di], tiles_x, dt % tiles_x, dt // tiles_x)
        if s.kind == "camera" and (getattr(s, "support", 0) & 4) and len(diff):
            # the camera tile cull's decision within FP32 noise of its threshold
            ok |= np.abs(oracle.tile_margin(g, s, dt, di, proj)) <= CULL_BAND
        assert ok.all(), (f"sensor {k}: {int((~ok).sum())} pairs differ outside the guard band, e.g. "
                          f"(tile, id, extra) {[(int(a), int(b), bool(j < len(extra))) for j, (a, b) in enumerate(zip(dt, di)) if not ok[j]][:5]}")
        # order: tile-major, then depth; within a tile consecutive entries may only invert
        # across an FP32 depth tie
        assert np.all(np.diff(t_gpu) >= 0), f"sensor {k}: tiles out of order"
        d = proj["rec"][:, 6][i_gpu]
        same = t_gpu[1:] == t_gpu[:-1]
        inv = same & (d[1:] < d[:-1] * (1 - 1e-6))
        assert not inv.any(), f"sensor {k}: depth order broken at {np.nonzero(inv)[0][:5]}"
        # where the pair sets agree, the sequences agree up to the tie reorders
        if len(diff) == 0:
            mism = int((i_gpu != i_ref).sum())
        else:
            mism = -1
        total[0] += len(key_gpu)
        total[1] += len(diff)
        total[2] += max(mism, 0)
        off += nt
    print("lists: pairs", total[0], "optional pairs differing", total[1], "tie reorders", total[2])
    return total
