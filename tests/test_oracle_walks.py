"""Pins for the oracle's Algorithm 1 / Algorithm 2 walks against closed forms,
invariants and finite differences.

Tolerances: |mean - exact| <= 3.5 SE + bias budget.  The budget covers the
polygon's sagitta and the eps-shell / backward-difference bias that Sec. 5.3
discusses (h = 10 eps leaves an O(eps/h) bias in du/dn).
"""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle, z_scores

Z = 3.5


def _check(mean, se, exact, rel_bias, abs_bias=0.0):
    bias = rel_bias * np.abs(exact) + abs_bias
    z = z_scores(mean, se, exact, 0.0)
    ok = np.abs(mean - exact) <= Z * se + bias
    assert ok.all(), (np.round(z, 2), mean, exact)


def _run(sc, W, differential=True, **over):
    pr = to_oracle(sc, **over)
    out = oracle.run_walks(pr, sc.query, W, differential=differential)
    n = sc.query.shape[0]
    m, se = est.point_mean_se(out["u_hat"], n, W)
    res = {"u": m, "u_se": se, "out": out}
    if differential:
        md, sed = est.point_mean_se(out["udot"], n, W)
        res.update(du=md, du_se=sed)
    return res


def test_laplace_never_uses_roulette():
    sc = scenes.disk_scene("screened_1", n_query=4)
    r = _run(sc, 256, sigma=0.0)
    assert np.all(r["out"]["kind"] == oracle.KIND_SHELL)


def test_offset_inside_shell_gives_zero_normal_derivative():
    # Sec. 5.3: with h < eps the nested walk stops at once and returns g(xbar),
    # so every du/dn estimate (and udot, for constant data) is exactly zero.
    sc = scenes.disk_scene("screened_1", n_query=6)
    r = _run(sc, 128, h=5e-4)
    o = r["out"]
    hit = o["kind"][:, 0] == oracle.KIND_SHELL
    assert hit.any()
    assert np.all(o["dudn"] == 0.0) and np.all(o["udot"] == 0.0)
    assert np.all(o["steps"][hit, 1] == 1)


def test_roulette_walks_have_zero_derivative():
    sc = scenes.disk_scene("screened_1", n_query=6)
    r = _run(sc, 256)
    o = r["out"]
    rr = o["kind"][:, 0] == oracle.KIND_ROULETTE
    assert rr.any()
    assert np.all(o["udot"][rr] == 0.0) and np.all(o["elem"][rr] == -1)


def test_walks_are_replayable_across_thread_counts():
    sc = scenes.disk_scene("screened_1", n_query=4)
    pr = to_oracle(sc)
    a = oracle.run_walks(pr, sc.query, 64, differential=True, threads=1)
    b = oracle.run_walks(pr, sc.query, 64, differential=True, threads=4)
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True)
    # a walk's id alone fixes its path: running a subset with the matching base reproduces it
    c = oracle.run_walks(pr, sc.query[2:3], 64, differential=True, walk_id_base=2 * 64)
    assert np.array_equal(c["u_hat"], a["u_hat"][128:192])


def test_disk_screened_constant_data_closed_form():
    sc = scenes.disk_scene("screened_1", n_query=12)
    r = _run(sc, 8192)
    u, du = cf.disk_screened_const(sc.query, 1.0, 4.0)
    _check(r["u"], r["u_se"], u, 2e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.01)


def test_disk_restricted_linear_data_has_zero_derivative():
    # u = x exactly; udot = (dg/dn - du/dn) V_n = 0.  Dropping the dg/dn term of
    # Eq. (boundary_deriv_restricted) would give -n_x V_n instead.
    sc = scenes.disk_scene("laplace_x", n_query=12)
    r = _run(sc, 8192)
    _check(r["u"], r["u_se"], sc.query[:, 0], 0.0, 2e-3)
    _check(r["du"], r["du_se"], np.zeros_like(r["du"]), 0.0, 0.03)
    # the two halves of the boundary term are each far from zero
    o = r["out"]
    assert np.abs(o["dudn"]).mean() > 0.3


def test_disk_mapped_data_closed_form():
    sc = scenes.disk_scene("mapped_cos", n_query=12)
    r = _run(sc, 8192)
    u, du = cf.disk_mapped_cos(sc.query, 1.0)
    _check(r["u"], r["u_se"], u, 2e-3, 1e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.01)


def test_disk_mapped_data_parameters_closed_form():
    # Eq. (boundary_deriv_mapped) with a nonzero data derivative: g = c cos t + s sin t
    # with c, s parameters; du/dc = x/R and du/ds = y/R come from the sum over the hit
    # element's vertices of w_a dg_a/dtheta alone.  A dropped weight, a transposed
    # [parameter][vertex] index or a sign error in that sum breaks these two columns.
    sc = scenes.disk_scene("mapped_data", n_query=12)
    r = _run(sc, 8192)
    u, du = cf.disk_mapped_linear(sc.query, 1.0, sc.meta["c"], sc.meta["s"])
    _check(r["u"], r["u_se"], u, 2e-3, 1e-3)
    # the data columns carry no 1/h noise: a tight bias budget (polygon interpolation)
    _check(r["du"][:, -2:], r["du_se"][:, -2:], du[:, -2:], 4e-3, 1e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.01)
    # the data columns are the dg term alone, walk by walk: each equals the hit
    # element's interpolated cos / sin (V_n = 0 for c and s)
    o = r["out"]
    hit = o["elem"] >= 0
    e = o["elem"][hit]
    w1 = o["bary"][hit, 0]
    t = sc.meta["t"]
    a, b = sc.elem[e, 0], sc.elem[e, 1]
    want_c = (1 - w1) * np.cos(t[a]) + w1 * np.cos(t[b])
    want_s = (1 - w1) * np.sin(t[a]) + w1 * np.sin(t[b])
    assert np.allclose(o["udot"][hit, -2], want_c, atol=1e-12)
    assert np.allclose(o["udot"][hit, -1], want_s, atol=1e-12)


def test_disk_source_closed_forms():
    for sigma, f, g in [(0.0, 1.0, 0.5), (3.0, 2.0, 1.0)]:
        sc = scenes.disk_scene("screened_1", n_query=8)
        sc.g_vert = np.full(sc.vert.shape[0], g)
        r = _run(sc, 8192, sigma=sigma, f=f)
        u, du = cf.disk_screened_const(sc.query, 1.0, sigma, g=g, f=f)
        _check(r["u"], r["u_se"], u, 3e-3, 1e-3)
        _check(r["du"][:, :3], r["du_se"][:, :3], du[:, :3], 0.08, 0.01)


def test_harmonic_field_on_star_domain():
    # sigma = 0, g = x^2 - y^2 + 0.3 xy (harmonic): u = g everywhere, udot = 0
    st = scenes.star_box_scene(n_seg=512, n_query=8, walks=1)
    st.data = "field"
    st.field = np.array([0.1, 0, 0, 0, 1.0, -1.0, 0, 0.15, 0, 0])
    st.sigma = 0.0
    rng = np.random.default_rng(5)
    ang = rng.uniform(0, 2 * np.pi, 8)
    st.query = np.stack([0.6 * np.cos(ang), 0.6 * np.sin(ang)], 1)
    r = _run(st, 4096)
    _check(r["u"], r["u_se"], cf.harmonic_field(st.query, st.field), 0.0, 3e-3)
    _check(r["du"], r["du_se"], np.zeros_like(r["du"]), 0.0, 0.02)


@pytest.mark.parametrize("sigma,f", [(1.0, 0.0), (1.0, 0.5), (0.0, 1.0)])
def test_ball_closed_form(sigma, f):
    sc = scenes.ball_scene(freq=12, n_query=6, sigma=sigma, f=f)
    r = _run(sc, 2048)
    u, du = cf.ball_screened_const(sc.query, 1.0, sigma, g=1.0, f=f)
    _check(r["u"], r["u_se"], u, 6e-3, 1e-3)
    _check(r["du"], r["du_se"], du, 0.1, 0.02)


def test_shape_derivative_matches_central_differences():
    # Sec. 5.1: the differential estimate and finite differences of the forward
    # estimator agree in expectation.  Irregular 10-gon, sigma = 2, one point.
    base = np.array([1.0, 0.8, 1.1, 0.9, 1.2, 0.85, 1.0, 0.95, 1.15, 0.8])
    t = 2 * np.pi * np.arange(10) / 10
    vert = np.stack([base * np.cos(t), base * np.sin(t)], 1)
    elem = np.stack([np.arange(10), (np.arange(10) + 1) % 10], 1).astype(np.int32)
    jac = np.zeros((10, 2, 2))
    jac[3, :, 0] = [np.cos(t[3]), np.sin(t[3])]     # radial motion of vertex 3
    jac[7, :, 1] = [1.0, 0.0]                       # x-motion of vertex 7
    g = 1.0 + 0.5 * np.sin(t)
    xq = np.array([[0.35, 0.2]])
    common = dict(elem=elem, data_kind="mapped", g_vert=g, sigma=2.0, eps=1e-4, h=2e-3, K=1)
    pr = oracle.Problem(vert=vert, jac=jac, **common)
    W = 200000
    o = oracle.run_walks(pr, xq, W, differential=True)
    md, sed = est.point_mean_se(o["udot"], 1, W)
    dlt = 0.03
    for j in range(2):
        vals = []
        for s in (+1, -1):
            pv = oracle.Problem(vert=vert + s * dlt * jac[:, :, j], **common)
            ov = oracle.run_walks(pv, xq, W, differential=False, walk_id_base=10 ** 7)
            vals.append(ov["u_hat"])
        fd = (vals[0] - vals[1]) / (2 * dlt)
        fd_mean, fd_se = fd.mean(), fd.std(ddof=1) / np.sqrt(W)
        z = abs(md[0, j] - fd_mean) / np.sqrt(sed[0, j] ** 2 + fd_se ** 2)
        assert z < 4.0 or abs(md[0, j] - fd_mean) < 0.05 * abs(fd_mean), (j, md[0, j], fd_mean, z)
