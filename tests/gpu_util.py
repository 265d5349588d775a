"""Helpers for the GPU parity tests: run a frame through libsplat and compare with
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_2411_16816_gb300.render import Frame, gaussians_to_device

DEV = torch.device("cuda:0")

TOL_FEAT = 1e-4     # absolute, rendered features / colour
TOL_RANGE = 1e-4    # relative, expected and median range
TOL_GRAD = 1e-3     # relative


def run(g, sensors, keep_state=True, capacity=None):
    gd = gaussians_to_device(g, DEV)
    fr = Frame(sensors, len(g["opacities"]), g["features"].shape[1], DEV, capacity=capacity)
    out = fr.forward(gd, keep_state=keep_state)
    torch.cuda.synchronize()
    return fr, gd, out


def per_sensor(fr, out, key, kind):
    return [v.cpu().numpy().reshape(v.shape[0] * v.shape[1], *v.shape[2:]) for v in fr.split(out[key], kind)]


def check_render(fr, out, g, sensors, sel=None, max_marginal=0.02):
    """Compare every sensor's outputs with the oracle (on the selected ray indices)."""
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
        ref = oracle.render(g, s, sel=idx)
        ok = ~ref["marginal"]
        stats.append(1 - ok.mean())
        assert ok.mean() >= 1 - max_marginal, f"sensor {k}: marginal fraction {1 - ok.mean()}"
        take = (lambda a: a) if idx is None else (lambda a: a[idx])
        if s.kind == "camera":
            F, T = take(cams[ci]), take(camT[ci])
            ci += 1
            np.testing.assert_allclose(F[ok], ref["F"][ok], atol=TOL_FEAT, rtol=0, err_msg=f"camera {k} features")
            np.testing.assert_allclose(T[ok], ref["T"][ok], atol=TOL_FEAT, rtol=0, err_msg=f"camera {k} T")
        else:
            F, De, Dm, A = take(lids[li]), take(lre[li]), take(lrm[li]), take(lal[li])
            li += 1
            np.testing.assert_allclose(F[ok], ref["F"][ok], atol=TOL_FEAT, rtol=0, err_msg=f"lidar {k} features")
            np.testing.assert_allclose(A[ok], ref["alpha"][ok], atol=TOL_FEAT, rtol=0, err_msg=f"lidar {k} alpha")
            np.testing.assert_allclose(De[ok], ref["range_exp"][ok], rtol=TOL_RANGE, atol=TOL_RANGE,
                                       err_msg=f"lidar {k} expected range (m)")
            np.testing.assert_allclose(Dm[ok], ref["range_med"][ok], rtol=TOL_RANGE, atol=1e-5,
                                       err_msg=f"lidar {k} median range")
    return stats


def upstream(fr, sensors, g, seed, with_T=True):
    """Random upstream gradients, zero on the oracle's marginal rays."""
    rng = np.random.default_rng(seed)
    C = g["features"].shape[1]
    grads, per = {}, []
    cam_F, cam_T, lid_F, lid_D, lid_A = [], [], [], [], []
    for s in sensors:
        ref = oracle.render(g, s)
        keep = (~ref["marginal"]).astype(np.float64)
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
    f32 = lambda xs: torch.as_tensor(np.concatenate(xs).astype(np.float32), device=DEV)
    if cam_F:
        grads["cam_feat"], grads["cam_T"] = f32(cam_F), f32(cam_T)
    if lid_F:
        grads["lid_feat"], grads["lid_range_exp"], grads["lid_alpha"] = f32(lid_F), f32(lid_D), f32(lid_A)
    return grads, per


def oracle_grads(g, sensors, per):
    tot = None
    for s, u in zip(sensors, per):
        if s.kind == "camera":
            r = oracle.render_backward(g, s, u["gF"], u["gT"])
        else:
            r = oracle.render_backward(g, s, u["gF"], None, u["gD"], u["gA"])
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
