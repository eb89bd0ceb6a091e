"""Shared test helpers: turn a generated scene into an oracle problem."""
from __future__ import annotations

import numpy as np

import oracle


def to_oracle(sc, **over) -> "oracle.Problem":
    kw = dict(vert=sc.vert, elem=sc.elem, jac=sc.jac, data_kind=sc.data, g_vert=sc.g_vert,
              dg_vert=sc.dg_vert, field=sc.field, sigma=sc.sigma, f=sc.f, eps=sc.eps, h=sc.h,
              K=sc.K, seed=sc.seed, neumann=sc.neumann, neumann_h=sc.neumann_h)
    kw.update(over)
    return oracle.Problem(**kw)


def z_scores(est, se, ref, bias=0.0):
    """|est - ref| / sqrt(se^2 + bias^2) elementwise."""
    est, se, ref = np.asarray(est), np.asarray(se), np.asarray(ref)
    return np.abs(est - ref) / np.sqrt(se ** 2 + np.asarray(bias) ** 2 + 1e-300)
