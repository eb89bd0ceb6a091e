"""Nested-walk control variate in the oracle, and the table's host logic.

Each nested walk from x_off = xbar - h n contributes u - (q n + t) . (x_end -
x_off) to the backward difference du/dn = (g - u_off) / h.  Pins:
  * the tangential gradient of linear data c . x + c0 on a segment or a
    triangle is c minus its normal component (a property of the plane);
  * for any table the correction has mean zero: the same walks with and
    without it give du/dn estimates whose differences average to zero;
  * with the exact gradient of u = x (q = n_x, t = e_x - n_x n) the nested
    estimate leaves only the eps-shell offset, so du/dn's variance collapses
    while its mean stays at the closed form n_x.
A wrong sign, a wrong displacement (x_end - x0 instead of x_end - x_off) or a
dropped tangential term leaves the variance of the last check at its plain
level.
"""
import numpy as np

import oracle
from paper_2405_12964_gb300 import scenes
from oracle.cv import nested_cv_table, tangential_gradient
from tests.helpers import to_oracle


def test_tangential_gradient_of_linear_data():
    rng = np.random.default_rng(0)
    c = rng.normal(size=3)
    # segments
    v = rng.normal(size=(20, 2))
    e = np.arange(20, dtype=np.int32).reshape(10, 2)
    t = tangential_gradient(v, e, v @ c[:2] + 0.7)
    d = v[e[:, 1]] - v[e[:, 0]]
    n = np.stack([d[:, 1], -d[:, 0]], 1) / np.linalg.norm(d, axis=1)[:, None]
    want = c[None, :2] - (n @ c[:2])[:, None] * n
    assert np.allclose(t[:, :2], want, atol=1e-12) and np.all(t[:, 2] == 0)
    # triangles
    v = rng.normal(size=(30, 3))
    e = np.arange(30, dtype=np.int32).reshape(10, 3)
    t = tangential_gradient(v, e, v @ c - 1.3)
    N = np.cross(v[e[:, 1]] - v[e[:, 0]], v[e[:, 2]] - v[e[:, 0]])
    n = N / np.linalg.norm(N, axis=1)[:, None]
    want = c[None] - (n @ c)[:, None] * n
    assert np.allclose(t, want, atol=1e-10)
    tab = nested_cv_table(v, e, v @ c, np.arange(10.0))
    assert tab.shape == (10, 4) and tab.dtype == np.float32 and np.array_equal(tab[:, 0], np.arange(10.0))


def _dudn(sc, W, table=None):
    o = oracle.run_walks(to_oracle(sc, cv_elem=table), sc.query, W, differential=True)
    hit = o["elem"] >= 0
    return o, hit


def test_nested_correction_has_zero_mean():
    sc = scenes.disk_scene("mapped_cos", n_query=8)
    W = 1024
    rng = np.random.default_rng(1)
    tab = rng.normal(size=(sc.elem.shape[0], 4)) * 3.0
    o0, hit = _dudn(sc, W)
    o1, _ = _dudn(sc, W, tab)
    # identical walks: u and the boundary hits do not change, only du/dn
    assert np.array_equal(o0["u_hat"], o1["u_hat"]) and np.array_equal(o0["elem"], o1["elem"])
    # the corrected nested mean is the uncorrected one minus the table's terms
    assert np.array_equal(o0["u_plain"], o1["u_plain"]) and np.array_equal(o0["disp_n"], o1["disp_n"])
    assert np.allclose(o0["u_off"], o0["u_plain"]) and np.all(o0["disp_t"] == 0)
    q = np.where(hit, tab[np.maximum(o1["elem"], 0), 0], 0.0)
    assert np.allclose(o1["u_off"], o1["u_plain"] - q * o1["disp_n"] - o1["disp_t"], atol=1e-12)
    d = (o1["dudn"] - o0["dudn"])[hit]
    assert d.std() > 1.0                       # the correction is not trivially zero
    z = d.mean() / (d.std(ddof=1) / np.sqrt(d.size))
    assert abs(z) < 4.5, z


def test_exact_gradient_collapses_the_nested_variance():
    sc = scenes.disk_scene("laplace_x", n_query=16)
    W = 512
    v, e = sc.vert, sc.elem
    d = v[e[:, 1]] - v[e[:, 0]]
    n = np.stack([d[:, 1], -d[:, 0]], 1) / np.linalg.norm(d, axis=1)[:, None]
    n *= np.sign(((v[e[:, 0]] + v[e[:, 1]]) * n).sum(1))[:, None]        # outward: the walk's oriented normal
    tab = nested_cv_table(v, e, v[:, 0], n[:, 0]).astype(np.float64)
    o0, hit = _dudn(sc, W)
    o1, _ = _dudn(sc, W, tab)
    nx = o0["normal"][hit, 0]                                           # closed form du/dn of u = x
    r0, r1 = o0["dudn"][hit] - nx, o1["dudn"][hit] - nx
    ratio = r1.var() / r0.var()
    assert ratio < 0.05, ratio
    assert abs(r1.mean()) < 4.5 * r1.std() / np.sqrt(r1.size) + 0.05 # eps/h shell bias at most
