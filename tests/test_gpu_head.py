"""GPU parity of the per-ray lidar decoder (Sec. 3.3, App. B) against the FP64 head
oracle, and the gain of a decoder trained by these kernels on rays the rasterizer
renders over the plain composited channels."""
import math

import numpy as np
import pytest
import torch

from oracle import head as H
from paper_2411_16816_gb300 import scenes
from paper_2411_16816_gb300.head import PlainChannels, RayHead, flatten, head_inputs, render_lidar_decoded, unflatten
from paper_2411_16816_gb300.render import Frame, gaussians_to_device

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _bf16_params(head: RayHead) -> dict:
    """The parameters the decoder actually uses: BF16-rounded weights, FP32 biases."""
    p = unflatten(head.params.cpu().numpy())
    return {k: (H.bf16_round(v) if k.startswith("W") else v.astype(np.float64)) for k, v in p.items()}


def _data(R, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(R, 32)).astype(np.float32)
    return x, rng.uniform(size=R).astype(np.float32), (rng.uniform(size=R) < 0.3).astype(np.float32)


def test_forward_matches_oracle():
    head = RayHead(scenes.head_init_params(11), DEV)
    x, _, _ = _data(1000, 1)
    out = head.forward(torch.as_tensor(x, device=DEV)).cpu().numpy()
    ref = H.forward(x.astype(np.float64), _bf16_params(head))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-5)


def test_training_gradients_and_input_gradient_match_oracle():
    head = RayHead(scenes.head_init_params(12), DEV)
    x, yi, yd = _data(777, 2)      # not a multiple of the 128-ray tile
    tx = torch.as_tensor(x, device=DEV)
    dx = torch.empty_like(tx)
    head.grad.zero_()
    head.loss.zero_()
    head.accumulate(tx, torch.as_tensor(yi, device=DEV), torch.as_tensor(yd, device=DEV), dx)
    torch.cuda.synchronize()
    loss, g, gx = H.loss_backward(x.astype(np.float64), _bf16_params(head), yi, yd, want_dx=True)
    assert head.loss.item() == pytest.approx(loss, rel=1e-4)
    got = unflatten(head.grad.cpu().numpy())
    for k in H.ORDER:
        rel = np.linalg.norm(got[k] - g[k]) / np.linalg.norm(g[k])
        assert rel < 1e-3, (k, rel)
        np.testing.assert_allclose(got[k], g[k], atol=1e-3 * np.abs(g[k]).max() + 1e-7, rtol=0, err_msg=k)
    np.testing.assert_allclose(dx.cpu().numpy(), gx, atol=1e-3 * np.abs(gx).max(), rtol=0)


def _near_relu_decision(x, p, rel=3e-5):
    """Rays with a pre-activation within `rel` of the sum of its terms' magnitudes of 0:
    there the FP32 split products and the FP64 oracle may take different ReLU branches,
    and the input gradient of that ray may differ by a whole unit's term."""
    x = x.astype(np.float64)
    W1, b1, W2, b2 = (p[k].astype(np.float64) for k in ("W1", "b1", "W2", "b2"))
    z1 = x @ W1 + b1
    s1 = np.abs(x) @ np.abs(W1) + np.abs(b1)
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    s2 = h1 @ np.abs(W2) + np.abs(b2)
    return (np.abs(z1) < rel * s1).any(axis=1) | (np.abs(z2) < rel * s2).any(axis=1)


def test_training_gradients_over_many_tiles_per_block_match_oracle():
    """60,001 rays: about three 128-ray tiles per block of the persistent grid (the weight
    gradients accumulate across a block's tiles), the last tile ragged.  The input gradient
    is compared on the rays whose ReLU decisions are all clear of FP32 noise."""
    head = RayHead(scenes.head_init_params(14), DEV)
    x, yi, yd = _data(60_001, 4)
    tx = torch.as_tensor(x, device=DEV)
    dx = torch.empty_like(tx)
    head.grad.zero_()
    head.loss.zero_()
    head.accumulate(tx, torch.as_tensor(yi, device=DEV), torch.as_tensor(yd, device=DEV), dx)
    torch.cuda.synchronize()
    p = _bf16_params(head)
    loss, g, gx = H.loss_backward(x.astype(np.float64), p, yi, yd, want_dx=True)
    assert head.loss.item() == pytest.approx(loss, rel=1e-4)
    got = unflatten(head.grad.cpu().numpy())
    for k in H.ORDER:
        rel = np.linalg.norm(got[k] - g[k]) / np.linalg.norm(g[k])
        assert rel < 1e-3, (k, rel)
        np.testing.assert_allclose(got[k], g[k], atol=1e-3 * np.abs(g[k]).max() + 1e-7, rtol=0, err_msg=k)
    near = _near_relu_decision(x, p)
    assert near.mean() < 0.02, near.mean()
    np.testing.assert_allclose(dx.cpu().numpy()[~near], gx[~near], atol=1e-3 * np.abs(gx).max(), rtol=0)


def test_adam_step_and_bf16_copy_match_oracle():
    head = RayHead(scenes.head_init_params(13), DEV, lr=1e-2)
    x, yi, yd = _data(512, 3)
    p64 = head.params.cpu().numpy().astype(np.float64)
    m64, v64 = np.zeros_like(p64), np.zeros_like(p64)
    for step in range(1, 4):
        head.grad.zero_()
        head.loss.zero_()
        tx = torch.as_tensor(x, device=DEV)
        head.accumulate(tx, torch.as_tensor(yi, device=DEV), torch.as_tensor(yd, device=DEV))
        g = head.grad.cpu().numpy().astype(np.float64)
        head.step_count += 1
        from paper_2411_16816_gb300 import _lib as L
        from paper_2411_16816_gb300.render import _stream, _vp
        L.call("splat_head_adam", _vp(head.params), _vp(head.grad), _vp(head.m), _vp(head.v), head.lr, 0.9, 0.999,
               1e-8, step, _vp(head.w_bf16), _vp(head.bias), _stream())
        H.adam(p64, g, m64, v64, head.lr, 0.9, 0.999, 1e-8, step)
        torch.cuda.synchronize()
        np.testing.assert_allclose(head.params.cpu().numpy(), p64, rtol=1e-5, atol=1e-7)
    # the BF16 weights are the round-to-nearest-even images of the FP32 masters
    masters = unflatten(head.params.cpu().numpy())
    w = np.concatenate([H.bf16_round(masters[k]).astype(np.float32).reshape(-1) for k in ("W1", "W2", "W3")])
    got = (head.w_bf16.cpu().numpy().astype(np.uint16).astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(got, w)
    b = np.concatenate([masters[k].reshape(-1) for k in ("b1", "b2", "b3")])
    assert np.array_equal(head.bias.cpu().numpy(), b)


def test_head_inputs_pack_features_and_ray_directions():
    g = scenes.driving_gaussians(20000, 5, channels=29)
    elev = scenes.nonuniform_elevations(32)
    lid = scenes.Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=512, az_res=2 * math.pi / 512,
                       eps2d=scenes.lidar_blur(elev, 2 * math.pi / 512))
    fr = Frame([lid], 20000, 29, DEV)
    out = fr.forward(gaussians_to_device(g, DEV))
    x = head_inputs(fr, 0, out["lid_feat"]).cpu().numpy()
    assert np.array_equal(x[:, :29], out["lid_feat"].cpu().numpy())
    phi = (np.arange(512) + 0.5) * np.float32(lid.az_res)
    om = np.asarray(elev, np.float32).astype(np.float64)
    P, O = np.meshgrid(phi, om)
    d = np.stack([np.cos(O) * np.cos(P), np.cos(O) * np.sin(P), np.sin(O)], -1).reshape(-1, 3)
    np.testing.assert_allclose(x[:, 29:], d, atol=2e-6)


def test_decoder_fused_into_the_lidar_forward_equals_the_unfused_path():
    """splat_render_lidar_head renders the sweep exactly as the lidar forward does and
    decodes every ray inside the raster epilogue: outputs equal render -> head_inputs ->
    head forward bit for bit, with and without the features written; moving sensor,
    non-uniform beams, ragged last azimuth tile."""
    g = scenes.driving_gaussians(60_000, 1007, channels=29)
    gd = gaussians_to_device(g, DEV)
    elev = scenes.nonuniform_elevations(64)
    res = 2 * math.pi / 1000
    v, w = scenes.ego_motion(np.eye(3), 15.0, 0.05)
    lid = scenes.Lidar(R=np.eye(3), t=np.zeros(3), beam_elev=elev, n_az=1000, az_res=res, sweep_time=0.1,
                       eps2d=scenes.lidar_blur(elev, res), lin_vel=v, ang_vel=w)
    head = RayHead(scenes.head_init_params(5), DEV)
    fr = Frame([lid], len(g["opacities"]), 29, DEV)
    ref = fr.forward(gd)
    want = head.forward(head_inputs(fr, 0, ref["lid_feat"]))
    fused = render_lidar_decoded(fr, gd, head)
    torch.cuda.synchronize()
    assert (ref["lid_alpha"] > 0.5).float().mean() > 0.3
    for k in ("lid_feat", "lid_range_exp", "lid_range_med", "lid_alpha"):
        assert torch.equal(fused[k], ref[k]), k
    assert torch.equal(fused["head"], want)
    bare = render_lidar_decoded(fr, gd, head, features=False)
    torch.cuda.synchronize()
    assert bare["lid_feat"] is None and torch.equal(bare["head"], want)
    # against the FP64 decoder oracle on a sample of rays
    x = head_inputs(fr, 0, ref["lid_feat"]).cpu().numpy().astype(np.float64)
    sel = np.random.default_rng(3).choice(x.shape[0], 500, replace=False)
    o = H.forward(x[sel], _bf16_params(head))
    np.testing.assert_allclose(fused["head"].cpu().numpy()[sel], o, rtol=1e-4, atol=1e-4)


# ----------------------------------------------------------------------------------
# Gain: decoder trained by these kernels on rendered rays vs plain composited channels
# ----------------------------------------------------------------------------------

def _sweeps(n_gauss=200_000, n_poses=5, seed=1004):
    """Lidar sweeps (64 beams x 1024, non-uniform, 100 ms) from poses 0.5 m apart along +x,
    rendering 29 feature channels.  Returns the scene on the device, the lidars, and per
    sweep the decoder inputs of its hit rays (alpha > 0.5) and the hit mask."""
    g = scenes.driving_gaussians(n_gauss, seed, channels=29)
    gd = gaussians_to_device(g, DEV)
    elev = scenes.nonuniform_elevations(64)
    res = 2 * math.pi / 1024
    lids, xs, masks = [], [], []
    for k in range(n_poses):
        v, w = scenes.ego_motion(np.eye(3), 15.0, 0.0)
        lid = scenes.Lidar(R=np.eye(3), t=np.array([-0.5 * k, 0.0, 0.0]), beam_elev=elev, n_az=1024, az_res=res,
                           sweep_time=0.1, eps2d=scenes.lidar_blur(elev, res), lin_vel=v, ang_vel=w)
        fr = Frame([lid], n_gauss, 29, DEV)
        out = fr.forward(gd, keep_state=False)
        x = head_inputs(fr, 0, out["lid_feat"])
        keep = out["lid_alpha"] > 0.5          # rays that hit something
        lids.append(lid)
        xs.append(x[keep])
        masks.append(keep)
    return gd, lids, xs, masks


def _bce(p, y):
    p = np.clip(p, 1e-4, 1 - 1e-4)
    return -np.mean(y * np.log(p) + (1 - y) * np.log(1 - p))


def test_trained_head_beats_plain_composited_channels():
    """App. B's decoder against the method without it:
    per-Gaussian intensity and ray-drop logit channels composited by the rasterizer and
    fitted through its own backward with Adam, for the same 1,500 steps and loss.  Scored
    on a held-out sweep: intensity RMSE, drop BCE and the drop decision against the
    noise-free probability."""
    gd, lids, xs, masks = _sweeps()
    tp = scenes.teacher_params(77)
    data = []
    for k, x in enumerate(xs):
        xn = x.cpu().numpy()
        yi, yd, pd = scenes.teacher_labels(xn[:, :29], xn[:, 29:], tp, seed=100 + k)
        data.append((x, torch.as_tensor(yi, device=DEV), torch.as_tensor(yd, device=DEV), xn, yi, yd, pd))
    train, test = data[:-1], data[-1]
    steps = 1500
    xtr = torch.cat([d[0] for d in train])
    yitr = torch.cat([d[1] for d in train])
    ydtr = torch.cat([d[2] for d in train])
    head = RayHead(scenes.head_init_params(21), DEV, lr=3e-3)
    perm_rng = torch.Generator(device=DEV).manual_seed(0)
    n = xtr.shape[0]
    B = 16384
    for step in range(steps):
        idx = torch.randint(0, n, (B,), device=DEV, generator=perm_rng)
        head.train_step(xtr[idx].contiguous(), yitr[idx].contiguous(), ydtr[idx].contiguous())
    o = head.forward(test[0]).cpu().numpy().astype(np.float64)
    yi_te, yd_te, pd_te = test[4], test[5], test[6]
    head_rmse = np.sqrt(np.mean((1 / (1 + np.exp(-o[:, 0])) - yi_te) ** 2))
    head_pd = 1 / (1 + np.exp(-o[:, 1]))
    # drop labels are Bernoulli draws: score the predicted probability (held-out BCE) and
    # its decision against the noise-free one (p_drop > 0.5)
    head_bce, head_acc = _bce(head_pd, yd_te), np.mean((head_pd > 0.5) == (pd_te > 0.5))

    # the method without the decoder: two per-Gaussian channels fitted through the rasterizer
    n_g = gd["means"].shape[0]
    base = PlainChannels(gd, n_g, DEV, lr=0.05)
    frames = [Frame([lid], n_g, 2, DEV) for lid in lids]
    for step in range(steps):
        k = step % len(train)
        base.step(frames[k], masks[k], train[k][1], train[k][2])
    out = base.render(frames[-1])
    s_i, s_d = PlainChannels.predict(out["lid_feat"][masks[-1]])
    s_i = s_i.cpu().numpy().astype(np.float64)
    s_d = s_d.cpu().numpy().astype(np.float64)
    base_rmse = np.sqrt(np.mean((s_i - yi_te) ** 2))
    base_bce, base_acc = _bce(s_d, yd_te), np.mean((s_d > 0.5) == (pd_te > 0.5))
    print(f"held-out rays {len(yi_te)}: head RMSE {head_rmse:.4f} drop BCE {head_bce:.4f} decision {head_acc:.4f}; "
          f"per-Gaussian channels RMSE {base_rmse:.4f} drop BCE {base_bce:.4f} decision {base_acc:.4f}")
    assert head_rmse < 0.7 * base_rmse
    assert head_bce < base_bce
    assert head_acc > base_acc
