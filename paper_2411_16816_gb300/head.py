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
