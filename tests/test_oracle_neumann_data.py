"""Pins for the oracle's Neumann-data term of the walk on stars (Sec. 3.4,
Eq. mixed_bvp with Robin coefficient 0 and data h = du/dn on the Neumann part;
the derivative problem of Sec. 4.2, Eq. mixed_bvp_deriv, has zero Neumann data,
so the data reaches du/dtheta only through the nested walks).

* One step: the mean of the sample over many walk ids is the integral of
  G_R(x, z) h over the Neumann boundary in the ball that x sees, divided by the
  share of directions into the domain (1/2 on a side), computed by quadrature
  from the oracle's own ball Green's function (whose step weight is pinned to
  its flux elsewhere): a flat side below a point, the point on the side, the
  quarter disk's right-angled corner of two Neumann radii (share 1/4), and
  the thermal slab, where the far face must not count (hidden behind the near
  face from below, behind the side from a point on it); and, on a side cut into
  segments of very different lengths with data on one segment only, the
  draw's probability proportional to each candidate's length (a uniform mesh
  would pass any draw); in 3D the same with data on the icosphere's largest
  and smallest triangle (areas 1.6x apart; a uniform draw misses the smaller
  by 4.7 SE); with screening (sigma = 4) the sample follows the screened ball's
  Green's function in 2D and 3D, far from the Laplace one.
* The data only adds to the estimate: the walks' paths do not depend on it,
  and each walk's u and udot are affine in it (superposition of two data sets).
* Whole walks against closed forms: u = b x + c (y^2 - x^2) on a square and
  b x + c (y^2 + z^2 - 2 x^2) on a cube with Neumann data 2c (u and du/dX = 0,
  at interior points and on the Neumann faces), a screened square (u = cosh(k y)
  + s sinh(k x), du/dX of the moving side), an annulus with data on the
  inner circle (u = a + b log r) and, in 3D on a curved part, the flow past an
  icosphere plus a point source q / r (data q / a^2 on the sphere).
Tolerances: 3.5 SE + a bias budget (eps-shell, polygon, mapped data).
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle import closed_forms as cf
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle

Z = 3.5


def _green(dim, t, R):
    vol = np.pi * R * R if dim == 2 else 4.0 / 3.0 * np.pi * R ** 3
    return oracle.source_weight(dim, 0.0, R, t / R) / vol


def _step_mean(prob, x, R, n, **kw):
    v = np.array([oracle.neumann_data_sample(prob, x, R, walk_id=i, step=1, **kw) for i in range(n)])
    return v.mean(), v.std() / np.sqrt(n)


def _check(mean, se, exact, rel_bias, abs_bias=0.0):
    ok = np.abs(mean - exact) <= Z * se + rel_bias * np.abs(exact) + abs_bias
    assert ok.all(), (np.round(np.abs(mean - exact) / (se + 1e-300), 2), mean, exact)


def _run(sc, W, differential=True):
    out = oracle.run_walks(to_oracle(sc), sc.query, W, differential=differential)
    n = sc.query.shape[0]
    m, se = est.point_mean_se(out["u_hat"], n, W)
    res = {"u": m, "u_se": se, "out": out}
    if differential:
        res["du"], res["du_se"] = est.point_mean_se(out["udot"], n, W)
    return res


def test_one_step_is_the_integral_over_a_flat_side():
    # h = 2c = 1 on the Neumann sides y = -1, 1; x at height s above y = -1, ball radius R
    R, s, n = 0.5, 0.3, 20000
    L = np.sqrt(R * R - s * s)
    sc = scenes.neumann_data_box_scene(2, c=0.5)
    pr = to_oracle(sc)
    m, se = _step_mean(pr, [0.1, -1 + s], R, n)
    want = quad(lambda q: _green(2, np.hypot(s, q), R), -L, L)[0]
    assert abs(m - want) <= Z * se, (m, se, want)
    # on the side (the bottom element under x = 0.1): the whole chord of the ball, over the share 1/2
    e = int(np.nonzero((sc.neumann == 1) & (sc.vert[sc.elem[:, 0], 0] <= 0.1) & (sc.vert[sc.elem[:, 1], 0] > 0.1)
                       & (sc.vert[sc.elem[:, 0], 1] == -1.0))[0][0])
    m, se = _step_mean(pr, [0.1, -1.0], R, n, on=e, n_on=[0.0, -1.0])
    want_on = 2 * 2 * quad(lambda q: _green(2, q, R), 0, R)[0]
    assert abs(want_on - 2 * R / np.pi) < 1e-9          # 2 int_0^R log(R/t) / pi dt = 2 R / pi
    assert abs(m - want_on) <= Z * se, (m, se, want_on)
    # 3D, inside: the disk of the face y = -1 in the ball
    sc3 = scenes.neumann_data_box_scene(3, c=0.5)
    m, se = _step_mean(to_oracle(sc3), [0.1, -1 + s, 0.05], R, 100000)
    want = quad(lambda r: _green(3, np.hypot(s, r), R) * 2 * np.pi * r, 0, L)[0]
    assert abs(want - 0.02) < 1e-12                      # (R - s)^2 / (2 R) for G = (1/t - 1/R) / 4 pi
    assert abs(m - want) <= Z * se, (m, se, want)


def test_one_step_sees_only_the_star():
    # the thermal slab [-0.5, 0.5] x [0.2, 0.3] with h = 1 on every slab element
    sc = scenes.thermal_scene(n_query=2)
    sc.neumann_h = sc.neumann.astype(np.float64)
    pr = to_oracle(sc)
    n = 20000
    # from below, R = 0.25 reaches the top face (at 0.2) too, hidden behind the underside
    R, s = 0.25, 0.1
    m, se = _step_mean(pr, [0.0, 0.1], R, n)
    L = np.sqrt(R * R - s * s)
    want = quad(lambda q: _green(2, np.hypot(s, q), R), -L, L)[0]
    hidden = quad(lambda q: _green(2, np.hypot(2 * s, q), R), -np.sqrt(R * R - 4 * s * s), np.sqrt(R * R - 4 * s * s))[0]
    assert hidden > 4 * Z * se
    assert abs(m - want) <= Z * se, (m, se, want, hidden)
    # on the underside (element 88, normal out of the domain (0, 1)), R = 0.15: the top face lies
    # behind the side; the underside's chord counts, over the share 1/2
    R = 0.15
    m, se = _step_mean(pr, [0.0155, 0.2], R, n, on=88, n_on=[0.0, 1.0])
    want = 2 * R / np.pi
    Lb = np.sqrt(R * R - 0.01)
    behind = 2 * quad(lambda q: _green(2, np.hypot(0.1, q), R), -Lb, Lb)[0]
    assert behind > 4 * Z * se
    assert abs(m - want) <= Z * se, (m, se, want, behind)


@pytest.mark.parametrize("dim", [2, 3])
def test_box_with_neumann_data_closed_form(dim):
    sc = scenes.neumann_data_box_scene(dim, c=0.5, b=0.3, n_query=6)
    q = sc.query.copy()
    face = q[:2].copy()
    face[:, 1] = [-1.0, 1.0]                              # on the Neumann faces y = -1, 1
    sc.query = np.concatenate([q, face])
    r = _run(sc, 2048)
    u, du = cf.neumann_data_box(sc.query, 0.5, 0.3)
    _check(r["u"], r["u_se"], u, 0.0, 4e-3)
    _check(r["du"], np.maximum(r["du_se"], np.median(r["du_se"], axis=0)), du, 0.0, 0.02)
    # without the data the walks estimate another function, far outside the error bars
    sc.neumann_h = None
    r0 = _run(sc, 2048, differential=False)
    assert np.max(np.abs(r0["u"] - u) / r["u_se"]) > 20


def test_screened_square_with_neumann_data_closed_form():
    sc = scenes.screened_neumann_data_box_scene(k=1.5, s=0.5, n_query=6)
    r = _run(sc, 2048)
    u, du = cf.screened_neumann_data_box(sc.query, 1.5, 0.5)
    _check(r["u"], r["u_se"], u, 3e-3, 2e-3)
    _check(r["du"], np.maximum(r["du_se"], np.median(r["du_se"], axis=0)), du, 0.08, 0.02)
    assert (r["out"]["kind"][:, 0] == oracle.KIND_ROULETTE).any()


def test_annulus_with_neumann_data_closed_form():
    sc = scenes.annulus_neumann_data_scene(n_query=6)
    r = _run(sc, 2048, differential=False)
    u = cf.annulus_log(sc.query, 1.0, 0.5)
    _check(r["u"], r["u_se"], u, 0.0, 3e-3)


def test_one_step_at_an_edge_takes_the_wedge_share():
    # the quarter disk's corner at the origin, where its two Neumann radii meet at a right angle:
    # a walk there sits on the x-axis element 144 (normal out of the domain (0, -1)) and the y-axis
    # element 143 ((-1, 0)); the share of directions into the domain is 1/4, and both radii's
    # chords of the ball count: 2 int_0^R G / (1/4) = 4 R / pi
    sc = scenes.quarter_disk_scene("field", n_query=2)
    sc.neumann_h = sc.neumann.astype(np.float64)
    pr = to_oracle(sc)
    assert np.allclose(sc.vert[sc.elem[144]], [[0, 0], [1 / 16, 0]])
    assert np.allclose(sc.vert[sc.elem[143]], [[0, 1 / 16], [0, 0]])
    R = 0.3
    m, se = _step_mean(pr, [0.0, 0.0], R, 20000, on=144, n_on=[0.0, -1.0], on2=143, n2=[-1.0, 0.0])
    want = 4 * R / np.pi
    assert abs(m - want) <= Z * se, (m, se, want)
    # as if the walk were on one side only: the share 1/2 halves it
    m1, se1 = _step_mean(pr, [0.0, 0.0], R, 20000, on=144, n_on=[0.0, -1.0])
    assert abs(m1 - want / 2) <= Z * se1, (m1, se1, want / 2)


def test_the_data_enters_linearly_and_leaves_the_walks_unchanged():
    # the data sample adds to the estimate and draws from its own block: the walks' paths, steps
    # and terminal elements do not depend on h, and each walk's estimate is affine in h
    sc = scenes.thermal_scene(n_query=4)
    rng = np.random.default_rng(7)
    h1 = np.where(sc.neumann == 1, rng.normal(size=len(sc.elem)), 0.0)
    h2 = np.where(sc.neumann == 1, rng.normal(size=len(sc.elem)), 0.0)
    runs = {}
    for name, hv in (("0", None), ("1", h1), ("2", h2), ("12", h1 + 2.0 * h2)):
        sc.neumann_h = hv
        runs[name] = oracle.run_walks(to_oracle(sc), sc.query, 32, differential=True)
    for k in ("kind", "steps", "elem"):
        for name in ("1", "2", "12"):
            assert np.array_equal(runs[name][k], runs["0"][k])
    u0, u1, u2, u12 = (runs[n]["u_hat"] for n in ("0", "1", "2", "12"))
    assert np.abs(u1 - u0).max() > 1e-3 and np.abs(u2 - u0).max() > 1e-3
    assert np.allclose(u12 - u0, (u1 - u0) + 2.0 * (u2 - u0), rtol=1e-9, atol=1e-12)
    d0, d1, d2, d12 = (runs[n]["udot"] for n in ("0", "1", "2", "12"))
    assert np.allclose(d12 - d0, (d1 - d0) + 2.0 * (d2 - d0), rtol=1e-9, atol=1e-9)


def test_sphere_with_neumann_data_closed_form():
    # a curved Neumann part in 3D carrying data: the flow past the icosphere (720 triangles) plus a
    # point source q / r, du/dn = q / a^2 on the sphere; du/dc (the flow's scale) keeps the flow.
    # The icosphere's area is 0.85 % below the sphere's, so its flux is too: a bias of about
    # 0.0085 q / r in u
    q = 0.2
    sc = scenes.sphere_flow_scene(n_query=6, q=q)
    r = _run(sc, 2048)
    u, du = cf.sphere_flow(sc.query, sc.meta["a"], q)
    rr = np.linalg.norm(sc.query, axis=1)
    _check(r["u"], r["u_se"], u, 0.0, 3e-3 + 0.01 * q / rr)
    _check(r["du"], r["du_se"], du, 0.0, 3e-3)
    # the same boundary values without the data on the sphere miss by more than 8 SE
    sc.neumann_h = None
    r0 = _run(sc, 2048, differential=False)
    assert np.max(np.abs(r0["u"] - u) / r0["u_se"]) > 8


def test_one_step_draws_elements_in_proportion_to_their_length():
    # a box whose bottom (the Neumann part) is cut into segments of very different lengths
    # (nodes at -1 + 2 (i / 12)^2); data 1 on one segment and 0 elsewhere: the mean of the step's
    # sample is the quadrature over that segment's chord alone only if every candidate is drawn
    # with probability proportional to its length (on a uniform mesh any draw would pass)
    n = 12
    xs = -1.0 + 2.0 * (np.arange(n + 1) / n) ** 2
    bottom = np.stack([xs[:-1], np.full(n, -1.0)], 1)
    sides = [np.array([[1.0, -1.0]]), np.array([[1.0, 1.0]]), np.array([[-1.0, 1.0]])]
    vert = np.concatenate([bottom] + sides, 0)
    nv = len(vert)
    elem = np.stack([np.arange(nv), (np.arange(nv) + 1) % nv], 1).astype(np.int32)
    neumann = np.zeros(nv, np.int32)
    neumann[:n] = 1
    x, R = np.array([-0.5, -0.75]), 0.6
    s = x[1] + 1.0
    L = np.sqrt(R * R - s * s)
    lengths = np.diff(xs)
    cand = np.nonzero((xs[1:] > x[0] - L) & (xs[:-1] < x[0] + L))[0]
    assert lengths[cand].max() > 5 * lengths[cand].min()
    for e in (cand[0], cand[len(cand) // 2], cand[-1]):
        h = np.zeros(nv)
        h[e] = 1.0
        pr = oracle.Problem(vert=vert, elem=elem, data_kind="field", field=np.zeros(10), eps=1e-3,
                            neumann=neumann, neumann_h=h)
        m, se = _step_mean(pr, x, R, 20000)
        lo, hi = max(xs[e], x[0] - L), min(xs[e + 1], x[0] + L)
        want = quad(lambda q: _green(2, np.hypot(s, q - x[0]), R), lo, hi)[0]
        assert abs(m - want) <= Z * se, (e, lengths[e], m, se, want)


def test_one_step_draws_triangles_in_proportion_to_their_area():
    # 3D: the icosphere's triangles differ in area; data 1 on one triangle, x at 0.1 above its
    # centroid along its normal (it sees the whole triangle): the mean of the step's sample is
    # the integral of G_R over that triangle, which needs the draw proportional to area and
    # uniform points on the triangle
    from scipy.integrate import dblquad
    sc = scenes.sphere_flow_scene(n_query=2)
    v, el = sc.vert, sc.elem
    sph = np.nonzero(sc.neumann == 1)[0]
    a, b, c = v[el[sph, 0]], v[el[sph, 1]], v[el[sph, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    assert area.max() > 1.5 * area.min()
    R = 0.3
    for t in (sph[np.argmax(area)], sph[np.argmin(area)]):
        A, B, C = v[el[t]]
        nrm = np.cross(B - A, C - A)
        nrm /= np.linalg.norm(nrm)
        cen = (A + B + C) / 3
        if np.dot(nrm, cen) < 0:
            nrm = -nrm                                    # away from the sphere's centre
        x = cen + 0.1 * nrm
        h = np.zeros(len(el))
        h[t] = 1.0
        pr = to_oracle(sc, neumann_h=h)
        m, se = _step_mean(pr, x, R, 20000)
        jac = 2 * 0.5 * np.linalg.norm(np.cross(B - A, C - A))
        want = dblquad(lambda w, u: _green(3, np.linalg.norm(A + u * (B - A) + w * (C - A) - x), R) * jac,
                       0, 1, 0, lambda u: 1 - u)[0]
        assert abs(m - want) <= Z * se, (t, m, se, want)


@pytest.mark.parametrize("dim", [2, 3])
def test_one_step_uses_the_screened_green_function(dim):
    # sigma = 4: the sample weighs by the screened ball's Green's function (the oracle's source
    # weight over the ball's volume, pinned to its flux elsewhere), not the Laplace one
    sigma, R, s = 4.0, 0.5, 0.2
    sc = scenes.neumann_data_box_scene(dim, c=0.5)
    sc.sigma = sigma
    pr = to_oracle(sc)
    x = [0.1, -1 + s, 0.05][:dim]
    vol = np.pi * R * R if dim == 2 else 4.0 / 3.0 * np.pi * R ** 3
    G = lambda t, sg: oracle.source_weight(dim, sg, R, t / R) / vol
    L = np.sqrt(R * R - s * s)
    if dim == 2:
        want, lap = (quad(lambda q: G(np.hypot(s, q), sg), -L, L)[0] for sg in (sigma, 0.0))
    else:
        want, lap = (quad(lambda r: G(np.hypot(s, r), sg) * 2 * np.pi * r, 0, L)[0] for sg in (sigma, 0.0))
    m, se = _step_mean(pr, x, R, 40000)
    assert abs(lap - want) > 4 * Z * se
    assert abs(m - want) <= Z * se, (m, se, want, lap)
