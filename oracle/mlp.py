"""FP64 reference of the control-variate MLP (test infrastructure only).

Network (the contract both sides implement): features
    f(x, y) = (x, y, sin(pi x), sin(pi y), sin(pi (x + y)), 0 x 11)   (16 inputs)
four tanh hidden layers of width 64 and a linear output layer of width 8, of
which outputs 0 (u) and 1 (du/dn) are used.  Tensor-core arithmetic: every
matrix-product input (weights, layer inputs, back-propagated deltas) is
rounded to BF16 (round to nearest even); sums are exact here (FP64) and FP32 on
the GPU; biases, tanh and the loss stay in full precision, and tanh' = 1 - a^2
is taken from the activation as stored for the next product (BF16).  The
evaluation (u, its (x, y) gradient and du/dn) follows the same rules: the
gradient is the backward pass of output 0 through the same rounded products.

Flat parameter layout (FP32 master copy, 14088 values):
    W1 (64 x 16), b1 (64), W2 (64 x 64), b2, W3, b3, W4, b4, W5 (8 x 64), b5 (8)
with W[out][in] row-major.

Loss: L = (1/n) sum_s sum_k mask[s, k] (out[s, k] - target[s, k])^2, k in {0, 1}.
Adam (Kingma & Ba 2015) on the FP32 master parameters.
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
          ("W4", (64, 64)), ("b4", (64,)), ("W5", (8, 64)), ("b5", (8,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(a):
    """Round FP32 values to BF16 (nearest even) and return them as FP64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a32)
    if nan.any():
        out[nan] = np.nan
    return out


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, s in SHAPES:
        n = int(np.prod(s))
        out[name] = p[o:o + n].reshape(s)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def features(x):
    x = np.asarray(x, dtype=np.float64)
    f = np.zeros((x.shape[0], 16))
    f[:, 0] = x[:, 0]
    f[:, 1] = x[:, 1]
    f[:, 2] = np.sin(np.pi * x[:, 0])
    f[:, 3] = np.sin(np.pi * x[:, 1])
    f[:, 4] = np.sin(np.pi * (x[:, 0] + x[:, 1]))
    return f


def _ident(a):
    return np.asarray(a, dtype=np.float64)


def forward(params, x, rounding: bool = True):
    """Training-precision forward pass; returns outputs and the activations.
    rounding=False drops the BF16 rounding (the exact FP64 network)."""
    r = bf16 if rounding else _ident
    P = unpack(params)
    a = [features(x)]
    for l in range(1, 5):
        z = r(a[-1]) @ r(P[f"W{l}"]).T + P[f"b{l}"]
        a.append(np.tanh(z))
    out = r(a[-1]) @ r(P["W5"]).T + P["b5"]
    return out, a


def loss_and_grad(params, x, target, mask, rounding: bool = True):
    """Masked MSE and its gradient with respect to the flat parameters."""
    r = bf16 if rounding else _ident
    n = x.shape[0]
    out, a = forward(params, x, rounding)
    err = np.zeros_like(out)
    err[:, :2] = mask * (out[:, :2] - target)
    loss = float((err[:, :2] ** 2).sum() / n)
    P = unpack(params)
    g = {}
    delta = 2.0 * err / n                                    # dL/d out, (n, 8)
    g["W5"] = r(delta).T @ r(a[4])
    g["b5"] = delta.sum(0)
    back = r(delta) @ r(P["W5"])                             # (n, 64)
    for l in range(4, 0, -1):
        d = back * (1.0 - r(a[l]) ** 2)
        g[f"W{l}"] = r(d).T @ r(a[l - 1])
        g[f"b{l}"] = d.sum(0)
        if l > 1:
            back = r(d) @ r(P[f"W{l}"])
    return loss, pack(g)


def adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new params, m, v."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def eval_u(params, x, rounding: bool = True):
    """Evaluation: u head, its gradient with respect to (x, y), and the du/dn
    head, in the training arithmetic (rounding=False: the exact network)."""
    r = bf16 if rounding else _ident
    P = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    out, a = forward(params, x, rounding)
    back = np.zeros((x.shape[0], 8))
    back[:, 0] = 1.0                                         # d u / d out
    back = r(back) @ r(P["W5"])                              # d u / d a4
    for l in range(4, 0, -1):
        d = back * (1.0 - r(a[l]) ** 2)                      # d u / d z_l
        back = r(d) @ r(P[f"W{l}"])                          # d u / d a_{l-1}
    df = back[:, :5]
    c0, c1, c01 = np.pi * np.cos(np.pi * x[:, 0]), np.pi * np.cos(np.pi * x[:, 1]), np.pi * np.cos(np.pi * (x[:, 0] + x[:, 1]))
    gx = df[:, 0] + df[:, 2] * c0 + df[:, 4] * c01
    gy = df[:, 1] + df[:, 3] * c1 + df[:, 4] * c01
    return out[:, 0], np.stack([gx, gy], 1), out[:, 1]


def init_params(seed: int = 0):
    """Xavier-uniform weights, zero biases, FP32 values."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, s in SHAPES:
        if name.startswith("W"):
            fan_out, fan_in = s
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            w = rng.uniform(-lim, lim, size=s)
            if name == "W1":
                w[:, 5:] = 0.0
            if name == "W5":
                w[2:, :] = 0.0
            d[name] = w
        else:
            d[name] = np.zeros(s)
    return pack(d).astype(np.float32).astype(np.float64)
