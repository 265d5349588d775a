"""Per-ray lidar decoder (paper Sec. 3.3 and App. B): rendered features + ray direction
-> 64 -> 64 -> (intensity logit, ray-drop logit), BF16 weights with FP32 masters and
FP32 accumulation, trained with lambda_intens L2(intensity) + lambda_raydrop BCE.

Device memory comes from torch; the forward, the fused training pass, the input
packing and the Adam update all run in libsplat's kernels (splat_head_*).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from .render import _stream, _vp

ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")
SIZES = {"W1": 32 * 64, "b1": 64, "W2": 64 * 64, "b2": 64, "W3": 64 * 2, "b3": 2}
LAMBDA_INTENSITY = 1.0
LAMBDA_RAYDROP = 0.1


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k in ORDER])


def unflatten(flat) -> dict:
    flat = np.asarray(flat)
    out, off = {}, 0
    shapes = {"W1": (32, 64), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (64, 2), "b3": (2,)}
    for k in ORDER:
        out[k] = flat[off:off + SIZES[k]].reshape(shapes[k])
        off += SIZES[k]
    return out


class RayHead:
    """Decoder state on the device: FP32 masters, Adam moments, BF16 weights, biases."""

    def __init__(self, params: dict, device="cuda", lr=3e-3, betas=(0.9, 0.999), eps=1e-8):
        self.lib = L.load()
        self.device = torch.device(device)
        n = self.lib.splat_head_param_count()
        flat = flatten(params)
        assert flat.size == n
        self.params = torch.as_tensor(flat, device=self.device).clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.w_bf16 = torch.zeros(32 * 64 + 64 * 64 + 64 * 2, dtype=torch.int16, device=self.device)
        self.bias = torch.zeros(130, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.step_count = 0
        self.refresh()

    def refresh(self):
        """Write the BF16 weights and FP32 biases from the masters (an Adam step with lr 0)."""
        zero = torch.zeros_like(self.params)
        L.call("splat_head_adam", _vp(self.params), _vp(zero), _vp(torch.zeros_like(self.m)),
               _vp(torch.zeros_like(self.v)), 0.0, self.betas[0], self.betas[1], self.eps, 1, _vp(self.w_bf16),
               _vp(self.bias), _stream())

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        R = x.shape[0]
        out = torch.empty((R, 2), dtype=torch.float32, device=self.device) if out is None else out
        L.call("splat_head_forward", _vp(x), R, _vp(self.w_bf16), _vp(self.bias), _vp(out), _stream())
        return out

    def accumulate(self, x, y_int, y_drop, dx: torch.Tensor | None = None):
        """Adds the loss and its parameter gradients of one batch (no update)."""
        L.call("splat_head_train", _vp(x), x.shape[0], _vp(self.w_bf16), _vp(self.bias), _vp(y_int), _vp(y_drop),
               LAMBDA_INTENSITY, LAMBDA_RAYDROP, _vp(self.grad), _vp(self.loss), _vp(dx), _stream())

    def train_step(self, x, y_int, y_drop, dx: torch.Tensor | None = None):
        self.grad.zero_()
        self.loss.zero_()
        self.accumulate(x, y_int, y_drop, dx)
        self.step_count += 1
        L.call("splat_head_adam", _vp(self.params), _vp(self.grad), _vp(self.m), _vp(self.v), self.lr,
               self.betas[0], self.betas[1], self.eps, self.step_count, _vp(self.w_bf16), _vp(self.bias), _stream())
        return self.loss


def head_inputs(frame, lidar_index: int, feat: torch.Tensor) -> torch.Tensor:
    """Decoder inputs [rays][32] for one lidar of a Frame from its rendered features
    (29 channels): features followed by the unit ray direction."""
    R = feat.shape[0]
    x = torch.empty((R, 32), dtype=torch.float32, device=feat.device)
    c = frame.c_sensors[lidar_index]
    L.call("splat_head_inputs", ctypes.byref(c), _vp(feat.contiguous()), feat.shape[1], _vp(x), _stream())
    return x


class PlainChannels:
    """The decoder-free form of the lidar channels: one intensity logit and one ray-drop
    logit per Gaussian, alpha-composited along each ray by the rasterizer like any other
    feature (Eq. alpha blend), intensity = sigmoid(composited logit), drop probability =
    sigmoid(composited logit).  The channels are fitted through the rasterizer's own
    backward pass with Adam on the decoder's loss (App. B weights: lambda_intens L2 +
    lambda_raydrop BCE), so it is the method without the decoder trained the same way.

    frames: one single-lidar Frame (2 channels) per training sweep, all over the same
    Gaussians; geometry: the device tensors of the scene's means, scales, quats,
    opacities (and velocities) -- not trained; targets: per sweep (ray mask, intensity,
    drop label) on the device."""

    def __init__(self, geometry: dict, n: int, device="cuda", lr=0.05, betas=(0.9, 0.999), eps=1e-8):
        self.device = torch.device(device)
        self.g = {k: v for k, v in geometry.items() if k != "features"}
        self.channels = torch.zeros((n, 2), dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.channels)
        self.v = torch.zeros_like(self.channels)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.t = 0

    def scene(self) -> dict:
        return dict(self.g, features=self.channels)

    def render(self, frame, keep_state=False) -> dict:
        return frame.forward(self.scene(), keep_state=keep_state)

    @staticmethod
    def predict(feat: torch.Tensor):
        """(intensity, drop probability) from composited channels [rays][2]."""
        return torch.sigmoid(feat[:, 0]), torch.sigmoid(feat[:, 1])

    def step(self, frame, mask: torch.Tensor, y_int: torch.Tensor, y_drop: torch.Tensor) -> float:
        """One Adam step on one sweep's rays selected by `mask` (their targets y_int, y_drop
        are given for the selected rays, in ray order).  Returns the loss (device sync)."""
        out = self.render(frame, keep_state=True)
        F = out["lid_feat"]
        n = max(int(mask.sum().item()), 1)
        s_i, s_d = self.predict(F[mask])
        loss = LAMBDA_INTENSITY * ((s_i - y_int) ** 2).mean() + LAMBDA_RAYDROP * torch.nn.functional.binary_cross_entropy(
            s_d.clamp(1e-6, 1 - 1e-6), y_drop)
        dF = torch.zeros_like(F)
        dF[mask, 0] = LAMBDA_INTENSITY * 2.0 * (s_i - y_int) * s_i * (1 - s_i) / n
        dF[mask, 1] = LAMBDA_RAYDROP * (s_d - y_drop) / n
        grads = frame.backward(self.scene(), out, {"lid_feat": dF})["features"]
        self.t += 1
        b1, b2 = self.betas
        self.m.mul_(b1).add_(grads, alpha=1 - b1)
        self.v.mul_(b2).addcmul_(grads, grads, value=1 - b2)
        mh = self.m / (1 - b1 ** self.t)
        vh = self.v / (1 - b2 ** self.t)
        self.channels.addcdiv_(mh, vh.sqrt().add_(self.eps), value=-self.lr)
        return float(loss.item())


def render_lidar_decoded(frame, g: dict, head: RayHead, features: bool = True, prepared=None, out: dict | None = None,
                         stream=None) -> dict:
    """The frame's lidar sweeps rendered and decoded in one launch per frame
    (splat_render_lidar_head): the lidar outputs of Frame.forward plus out["head"]
    [rays][2] = (intensity logit, ray-drop logit) of every lidar ray, equal to
    head.forward(head_inputs(...)) bit for bit.  The scene must have 29 channels.
    `prepared` (the c_gaussians of an already projected and binned frame) skips the
    projection and binning; without `features` the rendered features are not written."""
    cg = frame.prepare(g, stream=stream) if prepared is None else prepared
    dev = frame.device
    R = frame.lid_rays
    if out is None:
        out = {"lid_feat": torch.empty((R, frame.channels), dtype=torch.float32, device=dev) if features else None,
               "lid_range_exp": torch.empty(R, dtype=torch.float32, device=dev),
               "lid_range_med": torch.empty(R, dtype=torch.float32, device=dev),
               "lid_alpha": torch.empty(R, dtype=torch.float32, device=dev),
               "head": torch.empty((R, 2), dtype=torch.float32, device=dev)}
    L.call("splat_render_lidar_head", ctypes.byref(cg), len(frame.sensors), frame.c_sensors, frame.c_proj(),
           frame.c_bins(), _vp(out.get("lid_feat")), _vp(out["lid_range_exp"]), _vp(out["lid_range_med"]),
           _vp(out["lid_alpha"]), _vp(out.get("lid_T")), _vp(out.get("lid_last")), _vp(head.w_bf16), _vp(head.bias),
           _vp(out["head"]), _stream(stream))
    return out
