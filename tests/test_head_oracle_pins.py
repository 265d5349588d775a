"""Pins of the FP64 head oracle (per-ray lidar decoder, Sec. 3.3 / App. B) against
library routines written independently of it: numpy matrix products for the forward,
central finite differences for the backward, torch.optim.Adam for the update and
torch's bfloat16 conversion for the weight rounding."""
import numpy as np
import pytest
import torch

from oracle import head as H
from paper_2411_16816_gb300 import scenes


def _params(seed=3):
    p = scenes.head_init_params(seed)
    rng = np.random.default_rng(seed)
    return {k: H.bf16_round(v + (rng.normal(0, 0.05, v.shape).astype(np.float32) if v.ndim == 1 else 0))
            for k, v in p.items()}


def _data(R=37, seed=4):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(R, 32))
    return x, rng.uniform(size=R), (rng.uniform(size=R) < 0.3).astype(np.float64)


def test_bf16_rounding_matches_torch():
    a = np.random.default_rng(0).normal(size=10000).astype(np.float32) * 10
    a[:4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.0 - 2 ** -8, 0.0]   # ties to even
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(H.bf16_round(a), ref)


def test_forward_matches_matrix_products():
    p = _params()
    x, _, _ = _data()
    h1 = np.maximum(x @ p["W1"] + p["b1"], 0)
    h2 = np.maximum(h1 @ p["W2"] + p["b2"], 0)
    np.testing.assert_allclose(H.forward(x, p), h2 @ p["W3"] + p["b3"], rtol=1e-12, atol=1e-12)


def test_loss_value_matches_definition():
    p = _params()
    x, yi, yd = _data()
    o = H.forward(x, p)
    s = 1 / (1 + np.exp(-o[:, 0]))
    bce = -(yd * np.log(1 / (1 + np.exp(-o[:, 1]))) + (1 - yd) * np.log(1 - 1 / (1 + np.exp(-o[:, 1]))))
    ref = 1.0 * np.mean((s - yi) ** 2) + 0.1 * np.mean(bce)
    loss, _, _ = H.loss_backward(x, p, yi, yd)
    assert loss == pytest.approx(ref, rel=1e-12)


def test_gradients_match_finite_differences():
    p = _params()
    x, yi, yd = _data(R=9)
    _, g, gx = H.loss_backward(x, p, yi, yd, want_dx=True)
    h = 1e-6
    for k in H.ORDER:
        num = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            num[idx] = (H.loss_backward(x, pp, yi, yd)[0] - H.loss_backward(x, pm, yi, yd)[0]) / (2 * h)
        np.testing.assert_allclose(g[k], num, rtol=1e-5, atol=1e-9, err_msg=k)
    numx = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        numx[idx] = (H.loss_backward(xp, p, yi, yd)[0] - H.loss_backward(xm, p, yi, yd)[0]) / (2 * h)
    np.testing.assert_allclose(gx, numx, rtol=1e-5, atol=1e-9)


def test_adam_matches_torch():
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=500)
    grads = [rng.normal(size=500) for _ in range(4)]
    t = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(500), np.zeros(500)
    for step, g in enumerate(grads, 1):
        opt.zero_grad()
        t.grad = torch.tensor(g)
        opt.step()
        H.adam(p, g, m, v, 3e-3, 0.9, 0.999, 1e-8, step)
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)
