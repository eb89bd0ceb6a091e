"""The control-variate network's tensor-core kernels against the FP64
reference (oracle/mlp.py: the network with BF16 product operands, exact
otherwise) on the same parameters: loss and gradient, Adam steps, evaluation
of u, d u / d x and du/dn; and that training fits.

Loss, gradient and evaluation are compared element by element against the
bounds oracle/mlp.py derives for an implementation that accumulates in FP32,
evaluates tanh and the features in FP32, stores BF16 product operands and takes
tanh' from the stored activation (kernel_grad_bound, eval_bound): every weight
and bias of every layer must lie within its own bound."""
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
    Lr, Gr, E, EL = ref.kernel_grad_bound(p, x.astype(np.float64), t, m)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss[0]) - Lr) <= EL, (float(loss[0]), Lr, EL)
    G, R, B = ref.unpack(g), ref.unpack(Gr), ref.unpack(E)
    for k in R:          # every weight and bias of every layer
        ratio = np.abs(G[k] - R[k]) / np.maximum(B[k], 1e-300)
        assert np.all(np.abs(G[k] - R[k]) <= B[k]), (k, ratio.max(), np.unravel_index(np.argmax(ratio), ratio.shape))
    used = np.abs(Gr) > 1e-2 * np.abs(Gr).max()
    print("n=%d: max |gpu - ref| / bound %.3f; median bound / |ref| %.4f"
          % (n, (np.abs(g - Gr) / np.maximum(E, 1e-300)).max(), np.median(E[used] / np.abs(Gr[used]))))


def test_adam_steps_match_reference(net_cls):
    # Adam on its own: the oracle's Adam applied to the gradient the network's kernel
    # returns at the same parameters (the kernel is deterministic: fixed-order partial
    # sums, so train_step sees the same gradient as loss_grad).  The gradient itself is
    # checked against the definition above.  Tolerance: FP32 evaluation of the update
    # (about ten roundings of a value of size <= lr / (1 - beta1^t)) and the FP32 store
    # of the parameters.
    p = ref.init_params(3)
    net = net_cls.ControlVariateNet(params=p.astype(np.float32))
    x, t, m = _data(512, 4)
    lr = 1e-3
    mom, vel = np.zeros_like(p), np.zeros_like(p)
    q = p.copy()
    for it in range(1, 4):
        g = net.loss_grad(x, t, m)[1].cpu().numpy().astype(np.float64)
        net.train_step(x, t, m, lr=lr)
        q, mom, vel = ref.adam(q, g, mom, vel, it, lr)
        got = net.params().cpu().numpy().astype(np.float64)
        tol = 4.0 * np.abs(q) * 2.0 ** -24 + 20 * 2.0 ** -24 * lr / (1 - 0.9 ** it)
        assert np.all(np.abs(got - q) <= tol), (it, (np.abs(got - q) / tol).max())
        q = got


def test_eval_matches_reference(net_cls):
    p = ref.init_params(5) * 2.0
    net = net_cls.ControlVariateNet(params=p.astype(np.float32))
    rng = np.random.default_rng(6)
    x = rng.uniform(-0.95, 0.95, size=(300, 2)).astype(np.float32)
    u, gu, q = (a.cpu().numpy() for a in net.eval(x))
    (ur, gr, qr), (Eu, Eg, Eq) = ref.eval_bound(p, x.astype(np.float64))
    for name, got, want, E in (("u", u, ur, Eu), ("du/dn", q, qr, Eq), ("grad u", gu, gr, Eg)):
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= E), (name, (err / E).max())


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
