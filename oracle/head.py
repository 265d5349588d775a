"""FP64 oracle of the per-ray lidar decoder (test infrastructure; see head_oracle.c).

Sec. 3.3: rendered features + ray direction -> small MLP -> intensity and ray-drop
probability; App. B: loss weights lambda_intens = 1.0, lambda_raydrop = 0.1.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib, _ptr

IN, HID, OUT = 32, 64, 2
SHAPES = {"W1": (IN, HID), "b1": (HID,), "W2": (HID, HID), "b2": (HID,), "W3": (HID, OUT), "b3": (OUT,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def _declare(L):
    P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    L.head_forward.restype = ctypes.c_int
    L.head_forward.argtypes = [I64] + [P] * 8
    L.head_loss_backward.restype = D
    L.head_loss_backward.argtypes = [I64] + [P] * 9 + [D, D] + [P] * 7
    L.head_adam.restype = ctypes.c_int
    L.head_adam.argtypes = [I64, P, P, P, P, D, D, D, D, I64]


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def forward(x, p: dict) -> np.ndarray:
    """Raw outputs (intensity logit, drop logit), shape (R, 2)."""
    L = lib()
    x = _d(x)
    R = x.shape[0]
    out = np.zeros((R, OUT))
    args = [_d(p[k]) for k in ORDER]
    L.head_forward(R, _ptr(x), *[_ptr(a) for a in args], _ptr(out))
    return out


def loss_backward(x, p: dict, y_int, y_drop, lam_i=1.0, lam_d=0.1, want_dx=False):
    """(loss, grads dict, dx or None) of lam_i mean (sigmoid(o0) - y_int)^2 +
    lam_d mean BCE(o1, y_drop)."""
    L = lib()
    x = _d(x)
    R = x.shape[0]
    args = [_d(p[k]) for k in ORDER]
    g = {k: np.zeros(SHAPES[k]) for k in ORDER}
    gx = np.zeros_like(x) if want_dx else None
    loss = L.head_loss_backward(R, _ptr(x), *[_ptr(a) for a in args], _ptr(_d(y_int)), _ptr(_d(y_drop)),
                                float(lam_i), float(lam_d), *[_ptr(g[k]) for k in ORDER], _ptr(gx))
    return loss, g, gx


def adam(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, lr, beta1, beta2, eps, step):
    """One Adam step in place on FP64 arrays."""
    L = lib()
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    L.head_adam(p.size, _ptr(p), _ptr(_d(g)), _ptr(m), _ptr(v), float(lr), float(beta1), float(beta2), float(eps),
                int(step))
