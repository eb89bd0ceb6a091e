"""The control-variate network's tensor-core kernels against the FP64
reference (oracle/mlp.py) on the same parameters: loss and gradient, Adam
steps, evaluation of u, d u / d x and du/dn; and that training fits."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net_cls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    return dwos


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 2)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], np.cos(x[:, 1])], 1).astype(np.float32)
    m = (rng.random((n, 2)) < 0.8).astype(np.float32)
    return x, t, m


@pytest.mark.parametrize("n", [64, 1000, 50000])
def test_loss_and_gradient_match_reference(net_cls, n):
    # 64: one partial tile; 1000: eight tiles; 50000: more tiles than CTAs, so each
    # CTA accumulates several tiles' weight gradients in TMEM
    p = ref.init_params(1) * 2.0
    net = net_cls.ControlVariateNet(params=p.astype(np.float32))
    x, t, m = _data(n, 2)
    loss, g = net.loss_grad(x, t, m)
    Lr, Gr = ref.loss_and_grad(p, x, t, m)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss[0]) - Lr) <= 1e-4 * abs(Lr)
    assert np.linalg.norm(g - Gr) <= 2e-3 * np.linalg.norm(Gr), np.linalg.norm(g - Gr) / np.linalg.norm(Gr)
    # per-layer agreement
    G, R = ref.unpack(g), ref.unpack(Gr)
    for k in R:
        assert np.linalg.norm(G[k] - R[k]) <= 5e-3 * np.linalg.norm(R[k]) + 1e-9, k


def test_adam_steps_match_reference(net_cls):
    p = ref.init_params(3)
    net = net_cls.ControlVariateNet(params=p.astype(np.float32))
    x, t, m = _data(512, 4)
    mom, vel = np.zeros_like(p), np.zeros_like(p)
    q = p.copy()
    for it in range(1, 4):
        net.train_step(x, t, m, lr=1e-3)
        _, Gr = ref.loss_and_grad(q, x, t, m)
        q, mom, vel = ref.adam(q, Gr, mom, vel, it, 1e-3)
        q = q.astype(np.float32).astype(np.float64)
    got = net.params().cpu().numpy().astype(np.float64)
    assert np.abs(got - q).max() <= 3e-5, np.abs(got - q).max()


def test_eval_matches_reference(net_cls):
    p = ref.init_params(5) * 2.0
    net = net_cls.ControlVariateNet(params=p.astype(np.float32))
    rng = np.random.default_rng(6)
    x = rng.uniform(-0.95, 0.95, size=(300, 2)).astype(np.float32)
    u, gu, q = (a.cpu().numpy() for a in net.eval(x))
    ur, gr, qr = ref.eval_u(p, x)
    # same BF16 rounding on both sides; FP32 accumulation order can move an
    # activation across a BF16 rounding boundary (2^-8 relative) now and then
    for got, want, tol in ((u, ur, 2e-3), (q, qr, 2e-3), (gu, gr, 5e-3)):
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max() / scale
        assert np.median(np.abs(got - want)) <= 1e-4 * scale


def test_training_fits_a_smooth_field(net_cls):
    net = net_cls.ControlVariateNet(seed=7)
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, size=(4096, 2)).astype(np.float32)
    t = np.stack([0.5 * np.sin(np.pi * x[:, 0]) * np.cos(x[:, 1]), x[:, 0] * x[:, 1]], 1).astype(np.float32)
    m = np.ones_like(t)
    first = float(net.train_step(x, t, m, lr=3e-3)[0])
    for _ in range(400):
        last = float(net.train_step(x, t, m, lr=3e-3)[0])
    assert last < 0.05 * first, (first, last)
