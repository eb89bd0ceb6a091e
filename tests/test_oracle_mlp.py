"""Pins for the FP64 control-variate MLP reference (oracle/mlp.py)."""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32) * 10 ** rng.uniform(-6, 6, 5000).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 1e-40], dtype=np.float32)])
    want = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 2))
    t = rng.normal(size=(n, 2))
    m = (rng.random((n, 2)) < 0.7).astype(float)
    return x, t, m


def test_exact_gradient_matches_central_differences():
    p = mlp.init_params(3) * 3.0       # larger weights: nonlinear regime
    x, t, m = _data(40, 1)
    L, g = mlp.loss_and_grad(p, x, t, m, rounding=False)
    rng = np.random.default_rng(2)
    idx = rng.choice(mlp.N_PARAM, size=60, replace=False)
    # include biases of every layer and the output layer's used rows
    idx = np.concatenate([idx, [1024, 1024 + 64 + 4096 + 5, mlp.N_PARAM - 8, mlp.N_PARAM - 7]])
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, x, t, m, rounding=False)[0] - mlp.loss_and_grad(pm, x, t, m, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_rounded_gradient_close_to_exact():
    p = mlp.init_params(4)
    x, t, m = _data(256, 5)
    _, g = mlp.loss_and_grad(p, x, t, m)
    _, ge = mlp.loss_and_grad(p, x, t, m, rounding=False)
    assert np.linalg.norm(g - ge) <= 0.03 * np.linalg.norm(ge)


def test_eval_gradient_matches_central_differences():
    p = mlp.init_params(6) * 2.0
    rng = np.random.default_rng(7)
    x = rng.uniform(-0.9, 0.9, size=(20, 2))
    u, gu, q = mlp.eval_u(p, x, rounding=False)
    h = 1e-6
    for k in range(2):
        d = np.zeros(2)
        d[k] = h
        fd = (mlp.eval_u(p, x + d, rounding=False)[0] - mlp.eval_u(p, x - d, rounding=False)[0]) / (2 * h)
        assert np.allclose(gu[:, k], fd, rtol=1e-6, atol=1e-8)
    out, _ = mlp.forward(p, x, rounding=False)
    assert np.allclose(u, out[:, 0]) and np.allclose(q, out[:, 1])


def test_adam_matches_torch():
    rng = np.random.default_rng(8)
    p = rng.normal(size=50)
    w = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for t in range(1, 6):
        g = rng.normal(size=50)
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = mlp.adam(p, g, m, v, t, 1e-2)
    assert np.allclose(p, w.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_masked_outputs_do_not_train_unused_rows():
    p = mlp.init_params(9)
    x, t, m = _data(64, 10)
    _, g = mlp.loss_and_grad(p, x, t, m)
    G = mlp.unpack(g)
    assert np.all(G["W5"][2:] == 0) and np.all(G["b5"][2:] == 0)
