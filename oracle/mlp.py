"""FP64 reference of the control-variate MLP (test infrastructure only).

Network (the contract both sides implement): features
    f(x, y) = (x, y, sin(pi x), sin(pi y), sin(pi (x + y)), 0 x 11)   (16 inputs)
four tanh hidden layers of width 64 and a linear output layer of width 8, of
which outputs 0 (u) and 1 (du/dn) are used.  The network's matrix products take
BF16 operands (BF16 weights and tensor-core products): every matrix-product
input (weights, layer inputs, back-propagated deltas) is rounded to BF16
(round to nearest even) and nothing else is; sums, biases, tanh, its
derivative tanh' = 1 - a^2 (of the activation a itself) and the loss are exact
here (FP64).  The gradient is the exact backward pass of that network with the
rounding treated as the identity.  The evaluation (u, its (x, y) gradient and
du/dn) follows the same rules.

kernel_grad_bound and eval_bound give, element by element, how far a GPU
implementation of this network may land from these values when it follows the
arithmetic model stated there (FP32 accumulation, FP32 elementwise functions,
BF16 stores, tanh' from the BF16-stored activation): an error analysis carried
through the layers, not a copy of any kernel's results.

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
        d = back * (1.0 - a[l] ** 2)
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
        d = back * (1.0 - a[l] ** 2)                         # d u / d z_l
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


# ---------------------------------------------------------------------------
# Error bounds for a tensor-core implementation.
#
# Arithmetic model (what the bound assumes of the implementation, and nothing
# else): every matrix product takes BF16-rounded operands, whose products are
# exact in FP32, and sums them in FP32 in any order (error at most 2 k u
# sum |terms| for k terms, u = 2^-24, allowing directed rounding in the adds);
# biases, tanh (<= 2 ulp), sin / cos of the features (<= 2 ulp), the loss
# residuals and tanh' = 1 - r(a)^2 of the BF16-stored activation r(a) are FP32;
# values are stored to BF16 by round-to-nearest before they enter a product;
# the bias gradients come out of the weight-gradient products (sums of the
# BF16-rounded deltas), and the per-CTA partial gradients are summed in FP32.
#
# Each rounding event is bounded as above and, following the probabilistic
# model of rounding errors (independent, zero mean; Higham & Mary, SIAM J.
# Sci. Comput. 41(5), 2019), a quantity's error is a sum of such bounded terms
# carried through the network linearly: its scale S is the root of the sum of
# the squared bounds times their coefficients.  By Hoeffding's inequality the
# error exceeds C S with probability at most 2 exp(-C^2 / 2), 3e-8 for C = 6;
# the bound on a result is C S.  A BF16 store of a value known to within C S
# equals the store of the exact value unless a rounding boundary lies that
# close (checked value by value); then it can differ by the incoming error
# plus one BF16 step.  The store of tanh' from r(a) instead of a is a known
# rounding term |r(a)^2 - a^2| per unit.
# ---------------------------------------------------------------------------
U32 = 2.0 ** -24
C_SIGMA = 6.0


def _ulp32(v):
    return np.abs(np.asarray(v, dtype=np.float64)) * U32 * 2.0 + 1e-45


def _bf16_step(v):
    """Distance from r(v) to its neighbours (the BF16 spacing at |v|)."""
    a = np.abs(bf16(np.asarray(v, dtype=np.float64))) + 1e-38
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def _store(v, S):
    """Error scale of the BF16 store of a value known as v within C S, against
    the store r(v) of the exact value."""
    v = np.asarray(v, dtype=np.float64)
    E = C_SIGMA * np.asarray(S, dtype=np.float64) + _ulp32(v)
    rv = bf16(v)
    near = (bf16(v + E) != rv) | (bf16(v - E) != rv)
    return np.where(near, np.sqrt(S ** 2 + _bf16_step(v) ** 2), 0.0)


def _product(A, SA, B, SB, k):
    """Error scale of the FP32-accumulated product of operands A + e_A, B + e_B
    (k terms per sum) against A @ B."""
    acc = 2.0 * k * U32 * ((np.abs(A) + C_SIGMA * SA) @ (np.abs(B) + C_SIGMA * SB))
    return np.sqrt((SA ** 2) @ (B ** 2) + (A ** 2) @ (SB ** 2) + (SA ** 2) @ (SB ** 2) + acc ** 2)


def _forward_bounds(params, x):
    """Definition values and error scales of the forward pass."""
    P = unpack(params)
    A = [features(x)]
    # the implementation forms x, y (FP32 inputs) and sin(pi .) of them in FP32 (<= 2 ulp, and
    # the FP32 argument: |d sin(pi t)/dt| <= pi); the padding columns are exact zeros
    S0 = np.zeros_like(A[0])
    S0[:, :2] = _ulp32(A[0][:, :2])
    S0[:, 2:5] = 4.0 * _ulp32(A[0][:, 2:5]) + 4.0 * U32 * np.pi
    rA = [bf16(A[0])]
    SrA = [_store(A[0], S0)]
    for l in range(1, 5):
        rW = bf16(P[f"W{l}"])
        z = rA[-1] @ rW.T + P[f"b{l}"]
        Sz = np.sqrt(_product(rA[-1], SrA[-1], rW.T, 0 * rW.T, rW.shape[1]) ** 2 + _ulp32(z) ** 2)
        a = np.tanh(z)
        Sa = np.sqrt(((1.0 - a ** 2) * Sz) ** 2 + (2.0 * _ulp32(a)) ** 2)
        A.append(a)
        rA.append(bf16(a))
        SrA.append(_store(a, Sa))
    rW5 = bf16(P["W5"])
    out = rA[-1] @ rW5.T + P["b5"]
    Sout = np.sqrt(_product(rA[-1], SrA[-1], rW5.T, 0 * rW5.T, 64) ** 2 + _ulp32(out) ** 2)
    return P, A, rA, SrA, out, Sout


def _delta_below(back, Sback, a, ra, Sra):
    """Value and error scale of delta = back (1 - a^2) when the implementation
    forms it from back' (scale Sback) and tanh' of the stored activation r(a')."""
    d = back * (1.0 - a ** 2)
    t_round = np.abs(ra ** 2 - a ** 2)                       # r(a) instead of a
    t_step = Sra * (2.0 * np.abs(ra) + C_SIGMA * Sra)         # r(a') instead of r(a)
    babs = np.abs(back) + C_SIGMA * Sback
    S = np.sqrt(((1.0 - a ** 2) * Sback) ** 2 + (babs * t_round) ** 2 + (babs * t_step) ** 2
                + (2.0 * U32 * babs) ** 2 + (4.0 * _ulp32(d)) ** 2)
    return d, S


def _backward_bounds(P, A, rA, SrA, delta5, S5, n_acc):
    """Gradients (definition) and their bounds C S given the output deltas."""
    g, E = {}, {}
    d, Sd = delta5, S5
    for l in range(5, 0, -1):
        rd = bf16(d)
        Srd = _store(d, Sd)
        g[f"W{l}"] = rd.T @ rA[l - 1]
        E[f"W{l}"] = C_SIGMA * _product(rd.T, Srd.T, rA[l - 1], SrA[l - 1], n_acc)
        # bias gradient: the definition sums the deltas, the model their BF16 stores
        g[f"b{l}"] = d.sum(0)
        acc = 2.0 * n_acc * U32 * (np.abs(rd) + C_SIGMA * Srd).sum(0)
        E[f"b{l}"] = C_SIGMA * np.sqrt((Srd ** 2).sum(0) + ((rd - d) ** 2).sum(0) + acc ** 2)
        if l == 1:
            break
        rW = bf16(P[f"W{l}"])
        back = rd @ rW
        Sback = _product(rd, Srd, rW, 0 * rW, rW.shape[0])
        d, Sd = _delta_below(back, Sback, A[l - 1], rA[l - 1], SrA[l - 1])
    return g, E


def kernel_grad_bound(params, x, target, mask, n_cta=152):
    """Loss, gradient (both the definition, as loss_and_grad), a bound on
    |gradient of an implementation following the arithmetic model - gradient|
    per parameter (flat layout) and a bound on its loss's error.  n_cta: number
    of FP32 partial sums the implementation reduces at the end."""
    x = np.asarray(x, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    n = x.shape[0]
    P, A, rA, SrA, out, Sout = _forward_bounds(params, x)
    err = np.zeros_like(out)
    err[:, :2] = mask * (out[:, :2] - target)
    Se = np.zeros_like(out)
    Se[:, :2] = mask * np.sqrt(Sout[:, :2] ** 2 + (2.0 * _ulp32(out[:, :2] - target)) ** 2)
    delta = 2.0 * err / n
    Sdelta = np.sqrt((2.0 * Se / n) ** 2 + (2.0 * _ulp32(delta)) ** 2)
    # every product over the samples accumulates in FP32, then n_cta partials are added
    g, E = _backward_bounds(P, A, rA, SrA, delta, Sdelta, n + n_cta)
    loss = float((err[:, :2] ** 2).sum() / n)
    # (e'^2 - e^2) = (e' - e)(e' + e) per residual, then an FP32 sum of n terms
    ce = C_SIGMA * Se[:, :2]
    E_loss = float((ce * (2.0 * np.abs(err[:, :2]) + ce)).sum() / n + 2.0 * n * U32 * loss)
    return loss, pack(g), pack(E), E_loss


def eval_bound(params, x):
    """u, d u / d(x, y) and du/dn (the definition, as eval_u) and bounds C S for
    an implementation following the arithmetic model."""
    x = np.asarray(x, dtype=np.float64)
    P, A, rA, SrA, out, Sout = _forward_bounds(params, x)
    n = x.shape[0]
    d5 = np.zeros((n, 8))
    d5[:, 0] = 1.0
    rW5 = bf16(P["W5"])
    back = d5 @ rW5
    Sback = 2.0 * 8 * U32 * np.abs(d5) @ np.abs(rW5)
    for l in range(4, 0, -1):
        d, Sd = _delta_below(back, Sback, A[l], rA[l], SrA[l])
        rd = bf16(d)
        Srd = _store(d, Sd)
        rW = bf16(P[f"W{l}"])
        back = rd @ rW
        Sback = _product(rd, Srd, rW, 0 * rW, rW.shape[0])
    df, Sdf = back[:, :5], Sback[:, :5]
    c0, c1 = np.pi * np.cos(np.pi * x[:, 0]), np.pi * np.cos(np.pi * x[:, 1])
    c01 = np.pi * np.cos(np.pi * (x[:, 0] + x[:, 1]))
    Sc = 8.0 * U32 * np.pi
    gx = df[:, 0] + df[:, 2] * c0 + df[:, 4] * c01
    gy = df[:, 1] + df[:, 3] * c1 + df[:, 4] * c01
    Sgx = np.sqrt(Sdf[:, 0] ** 2 + (Sdf[:, 2] * c0) ** 2 + (Sdf[:, 4] * c01) ** 2 + (Sc * df[:, 2]) ** 2
                  + (Sc * df[:, 4]) ** 2 + (4.0 * _ulp32(np.abs(df[:, 0]) + np.abs(df[:, 2] * c0) + np.abs(df[:, 4] * c01))) ** 2)
    Sgy = np.sqrt(Sdf[:, 1] ** 2 + (Sdf[:, 3] * c1) ** 2 + (Sdf[:, 4] * c01) ** 2 + (Sc * df[:, 3]) ** 2
                  + (Sc * df[:, 4]) ** 2 + (4.0 * _ulp32(np.abs(df[:, 1]) + np.abs(df[:, 3] * c1) + np.abs(df[:, 4] * c01))) ** 2)
    C = C_SIGMA
    return (out[:, 0], np.stack([gx, gy], 1), out[:, 1]), (C * Sout[:, 0], C * np.stack([Sgx, Sgy], 1), C * Sout[:, 1])
