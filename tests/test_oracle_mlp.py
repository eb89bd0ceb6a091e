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


def _fp32_model(p, x, t, m):
    """An FP32 implementation of the arithmetic model of kernel_grad_bound, written
    independently of it: BF16-rounded product operands, FP32 matmuls (NumPy's own
    accumulation order), FP32 tanh, tanh' from the BF16-stored activation, bias
    gradients summed from the BF16-stored deltas."""
    f = np.float32
    P = mlp.unpack(p)
    r = lambda v: mlp.bf16(np.asarray(v, f)).astype(f)
    acts = [mlp.features(x).astype(f)]
    for l in range(1, 5):
        z = r(acts[-1]) @ r(P[f"W{l}"]).T + P[f"b{l}"].astype(f)
        acts.append(np.tanh(z).astype(f))
    out = r(acts[-1]) @ r(P["W5"]).T + P["b5"].astype(f)
    d = np.zeros_like(out)
    d[:, :2] = f(2.0) * (m.astype(f) * (out[:, :2] - t.astype(f))) / f(x.shape[0])
    g = {}
    for l in range(5, 0, -1):
        g[f"W{l}"] = r(d).T @ r(acts[l - 1])
        g[f"b{l}"] = r(d).sum(0, dtype=f)
        if l > 1:
            d = (r(d) @ r(P[f"W{l}"])) * (f(1.0) - r(acts[l - 1]) ** 2)
    return mlp.pack(g)


@pytest.mark.parametrize("n,scale", [(40, 3.0), (700, 1.0)])
def test_kernel_bound_holds_for_an_fp32_implementation(n, scale):
    p = mlp.init_params(11) * scale
    x, t, m = _data(n, 12)
    L, g, E, EL = mlp.kernel_grad_bound(p, x, t, m)
    L0, g0 = mlp.loss_and_grad(p, x, t, m)
    assert np.array_equal(g, g0) and L == L0          # the bound reports the definition's values
    emu = _fp32_model(p, x, t, m)
    assert np.all(np.abs(emu - g) <= E), np.max(np.abs(emu - g) / (E + 1e-300))
    # it is needed: the FP32 implementation does differ from the definition
    assert np.abs(emu - g).max() > 0
    # and it is informative: plausible mistakes in an implementation fall outside it
    G = mlp.unpack(g)
    off = {k: o for k, o in zip(G, np.cumsum([0] + [G[k].size for k in G])[:-1])}
    big = lambda k: off[k] + int(np.argmax(np.abs(G[k]).reshape(-1)))
    for name, mistake in [("bias column dropped", lambda v: v.__setitem__(slice(off["b2"], off["b2"] + 64), 0.0)),
                          ("one weight 30 % off", lambda v: v.__setitem__(big("W3"), 1.3 * v[big("W3")])),
                          ("one weight with the wrong sign", lambda v: v.__setitem__(big("W1"), -v[big("W1")])),
                          ("output bias scaled", lambda v: v.__setitem__(off["b5"], 1.5 * v[off["b5"]]))]:
        bad = emu.copy()
        mistake(bad)
        assert np.any(np.abs(bad - g) > E), name


def test_eval_bound_holds_for_an_fp32_forward():
    p = mlp.init_params(13) * 2.0
    rng = np.random.default_rng(14)
    x = rng.uniform(-0.9, 0.9, size=(300, 2))
    (u, gu, q), (Eu, Egu, Eq) = mlp.eval_bound(p, x)
    u0, gu0, q0 = mlp.eval_u(p, x)
    assert np.array_equal(u, u0) and np.array_equal(gu, gu0) and np.array_equal(q, q0)
    f = np.float32
    P = mlp.unpack(p)
    r = lambda v: mlp.bf16(np.asarray(v, f)).astype(f)
    a = mlp.features(x).astype(f)
    for l in range(1, 5):
        a = np.tanh(r(a) @ r(P[f"W{l}"]).T + P[f"b{l}"].astype(f)).astype(f)
    out = r(a) @ r(P["W5"]).T + P["b5"].astype(f)
    assert np.all(np.abs(out[:, 0] - u) <= Eu) and np.all(np.abs(out[:, 1] - q) <= Eq)
