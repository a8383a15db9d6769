"""Pins of the surrogate network's fp64 oracle: library routines (torch's
bfloat16 rounding, GELU, MSE and its autograd gradient), finite differences and
closed forms."""
import math

import numpy as np
import torch

from oracle import mlp_oracle as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, size=5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), want)


def test_gelu_matches_torch_and_limits():
    z = np.linspace(-8, 8, 401)
    want = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64)).numpy()
    assert np.allclose(M.gelu(z), want, rtol=1e-12, atol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # derivative by central differences
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, rtol=1e-6, atol=1e-8)


def test_backward_matches_finite_differences():
    dims = [8, 16, 16, 8]
    rng = np.random.default_rng(2)
    p = rng.normal(size=M.param_count(dims)) * 0.4
    x = rng.normal(size=(5, 8))
    dy = rng.normal(size=(5, 8))
    g = M.backward(dims, p, x, dy, bf16=False)
    h = 1e-6
    for i in rng.choice(len(p), size=60, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fp = (M.forward(dims, p + e, x, bf16=False)[0] * dy).sum()
        fm = (M.forward(dims, p - e, x, bf16=False)[0] * dy).sum()
        assert abs((fp - fm) / (2 * h) - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_single_linear_layer_closed_form():
    dims = [8, 8]
    rng = np.random.default_rng(3)
    p = rng.normal(size=M.param_count(dims))
    x = rng.normal(size=(4, 8))
    dy = rng.normal(size=(4, 8))
    g = M.backward(dims, p, x, dy, bf16=False)
    W = p[:64].reshape(8, 8)
    b = p[64:]
    y, _ = M.forward(dims, p, x, bf16=False)
    assert np.allclose(y, x @ W.T + b)
    assert np.allclose(g[:64].reshape(8, 8), dy.T @ x)
    assert np.allclose(g[64:], dy.sum(axis=0))


def test_mse_matches_torch_autograd():
    rng = np.random.default_rng(4)
    y = rng.normal(size=(6, 8))
    t = rng.normal(size=(6, 8))
    loss, dy = M.mse(y, t, used=3)
    ty = torch.tensor(y[:, :3], requires_grad=True)
    tl = torch.nn.functional.mse_loss(ty, torch.tensor(t[:, :3]))
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12
    assert np.allclose(dy[:, :3], ty.grad.numpy()) and not dy[:, 3:].any()


def test_adamw_first_step_closed_form():
    # after one step from zero moments, m_hat / sqrt(v_hat) = sign(g)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 2e-3])
    lr, wd, eps = 1e-2, 0.1, 1e-12
    p1, m, v = M.adamw(p, g, np.zeros(3), np.zeros(3), lr, 0.9, 0.999, eps, wd, 1)
    assert np.allclose(p1, p - lr * (np.sign(g) + wd * p), rtol=0, atol=1e-9)
    # against torch.optim.AdamW on the same numbers, several steps
    tp = torch.tensor(p, requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=lr, betas=(0.9, 0.999), eps=eps, weight_decay=wd)
    q, m, v = p.copy(), np.zeros(3), np.zeros(3)
    for step in range(1, 6):
        gs = g * step
        q, m, v = M.adamw(q, gs, m, v, lr, 0.9, 0.999, eps, wd, step)
        tp.grad = torch.tensor(gs)
        opt.step()
    assert np.allclose(q, tp.detach().numpy(), rtol=1e-12, atol=1e-12)
