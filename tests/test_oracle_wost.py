"""Pins for the oracle's walk on stars (mixed Dirichlet / reflecting Neumann
boundaries; Sec. 3.4, Eq. mixed_bvp with Robin coefficient 0 and zero Neumann
data) and its differential walk, which nests at the Dirichlet shell only
(Sec. 4.2, Eq. mixed_bvp_deriv).

* The step weight is the flux of the ball's Green's function per unit solid
  angle: checked against the Green's function itself (finite differences of
  the oracle's source weight), not a retyped formula.
* Closed forms: a quarter disk (u = x^2 - y^2, Neumann radii; du/dR for field
  and mapped data), a screened strip (u = cosh(kx)/cosh(k), Neumann top and
  bottom; du/dL of the moving side), a strip with a source, a slit disk
  (u = sqrt(r) cos(phi/2), discontinuous across a two-sided Neumann slit with
  an open end: a walk that stepped across the slit, as it would with a radius
  not bounded by the slit's silhouette, lands on the other side's data), a
  cube with four Neumann faces (u = x, du/dX of the moving face), and the
  potential flow past an insulating cylinder (u = x (1 + a^2/r^2), a curved
  Neumann part whose silhouettes are the points where rays graze it) and
  past an insulating sphere in 3D (u = x (1 + a^3 / (2 r^3))).
* Walks never end on the Neumann part.
Tolerances: 3.5 SE + a bias budget (polygon / mesh, eps-shell and the O(h)
backward difference of Sec. 5.3).
"""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle

Z = 3.5


def _check(mean, se, exact, rel_bias, abs_bias=0.0):
    ok = np.abs(mean - exact) <= Z * se + rel_bias * np.abs(exact) + abs_bias
    assert ok.all(), (np.round(np.abs(mean - exact) / (se + 1e-300), 2), mean, exact)


def _run(sc, W, differential=True, **over):
    out = oracle.run_walks(to_oracle(sc, **over), sc.query, W, differential=differential)
    n = sc.query.shape[0]
    m, se = est.point_mean_se(out["u_hat"], n, W)
    res = {"u": m, "u_se": se, "out": out}
    if differential:
        res["du"], res["du_se"] = est.point_mean_se(out["udot"], n, W)
    return res


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.0, 0.5, 9.0])
def test_star_weight_is_the_flux_of_the_ball_green_function(dim, sigma):
    R = 0.7
    vol = np.pi * R ** 2 if dim == 2 else 4.0 / 3.0 * np.pi * R ** 3
    area = lambda r: 2 * np.pi * r if dim == 2 else 4 * np.pi * r * r
    G = lambda r: oracle.source_weight(dim, sigma, R, r / R) / vol
    for t in (0.05, 0.2, 0.45, 0.69):
        hh = 1e-6
        flux = -(G(t + hh) - G(t - hh)) / (2 * hh) * area(t)
        assert abs(oracle.star_weight(dim, sigma, t, R) - flux) < 1e-6
    assert abs(oracle.star_weight(dim, sigma, R, R) - oracle.alpha(dim, sigma, R)) < 1e-12
    assert abs(oracle.star_weight(dim, sigma, 1e-7, R) - 1.0) < 1e-5
    if sigma == 0:
        assert oracle.star_weight(dim, sigma, 0.3, R) == 1.0


@pytest.mark.parametrize("data", ["field", "mapped"])
def test_quarter_disk_closed_form(data):
    sc = scenes.quarter_disk_scene(data, n_query=8)
    r = _run(sc, 4096)
    u, du = cf.quarter_disk(sc.query, data)
    _check(r["u"], r["u_se"], u, 3e-3, 2e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.02)
    o = r["out"]
    # walks end on the Dirichlet arc (elements 0 .. 127), never on the Neumann radii
    assert np.all(o["elem"][o["kind"][:, 0] == oracle.KIND_SHELL] < 128)
    # the data-independent part: with field data the two halves of udot cancel
    if data == "field":
        assert np.abs(o["dudn"]).mean() > 0.3


def test_screened_strip_closed_form():
    sc = scenes.strip_scene(sigma=4.0, n_query=8)
    r = _run(sc, 4096)
    u, du = cf.strip(sc.query, 4.0)
    _check(r["u"], r["u_se"], u, 3e-3, 1e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.01)
    assert (r["out"]["kind"][:, 0] == oracle.KIND_ROULETTE).any()


def test_strip_with_source_closed_form():
    # the source samples a point of the star, counted only where the walk sees it
    sc = scenes.strip_scene(sigma=0.0, f=2.0, g=0.5, n_query=8)
    r = _run(sc, 4096)
    u, du = cf.strip(sc.query, 0.0, f=2.0, g=0.5)
    _check(r["u"], r["u_se"], u, 4e-3, 2e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.02)


def test_slit_disk_needs_the_silhouette_bound():
    sc = scenes.slit_disk_scene(n_query=10)
    r = _run(sc, 4096, differential=False)
    _check(r["u"], r["u_se"], cf.slit_sqrt(sc.query), 0.0, 8e-3)
    # walks above and below the slit see different data: the values straddle zero
    assert (r["u"] > 0.2).any() and (r["u"] < -0.2).any()


def test_cube_with_neumann_faces_closed_form():
    sc = scenes.cube_neumann_scene(n_query=6)
    r = _run(sc, 2048)
    u, du = cf.cube_linear(sc.query)
    _check(r["u"], r["u_se"], u, 0.0, 4e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.02)
    o = r["out"]
    dirichlet = np.nonzero(sc.neumann == 0)[0]
    hit = o["kind"][:, 0] == oracle.KIND_SHELL
    assert np.isin(o["elem"][hit], dirichlet).all()


def test_cube_with_neumann_faces_and_a_source():
    # the source's samples count only where x sees them through the star: in 3D, with a source
    # f = 1.5, u = x + f (1 - x^2) / 2 and du/dX = (x + 1) (f - 1) / 2
    sc = scenes.cube_neumann_scene(n_query=6, f=1.5)
    r = _run(sc, 2048)
    u, du = cf.cube_linear(sc.query, 1.5)
    _check(r["u"], r["u_se"], u, 0.0, 5e-3)
    _check(r["du"], r["du_se"], du, 0.08, 0.02)


def test_screened_cube_closed_form():
    # screened walks on stars in 3D (Russian roulette by the 3D star weight): -u'' + 4 u = 0
    # between the Dirichlet faces, u = sinh(2 x) / sinh(2)
    sc = scenes.cube_neumann_scene(n_query=6, sigma=4.0)
    r = _run(sc, 2048)
    u, du = cf.cube_screened(sc.query, 4.0)
    _check(r["u"], r["u_se"], u, 0.0, 4e-3)
    # du/dX is a rare-event estimate far from the moving face (roulette ends most walks first):
    # its SE is floored at the median over the points
    _check(r["du"], np.maximum(r["du_se"], np.median(r["du_se"], axis=0)), du, 0.08, 0.02)
    assert (r["out"]["kind"][:, 0] == oracle.KIND_ROULETTE).any()


def test_cylinder_flow_closed_form():
    # a curved Neumann part: an insulating circle in a box held at the potential flow past it,
    # u = x (1 + a^2/r^2); its silhouette points (where rays from x graze the circle) bound the
    # stars, and du/dc = u tests the data derivative through walks on stars
    sc = scenes.cylinder_flow_scene(n_query=6)
    r = _run(sc, 2048)
    u, du = cf.cylinder_flow(sc.query, sc.meta["a"])
    _check(r["u"], r["u_se"], u, 0.0, 2e-3)
    _check(r["du"], r["du_se"], du, 0.0, 2e-3)
    o = r["out"]
    dirichlet = np.nonzero(sc.neumann == 0)[0]
    hit = o["kind"][:, 0] == oracle.KIND_SHELL
    assert np.isin(o["elem"][hit], dirichlet).all()
    assert np.all(np.hypot(o["x_end"][:, 0], o["x_end"][:, 1]) >= sc.meta["a"] * np.cos(np.pi / 300) - 1e-9)


def test_sphere_flow_closed_form():
    # a curved Neumann part in 3D: an insulating icosphere (720 triangles) in a box held at the
    # potential flow past it, u = x (1 + a^3 / (2 r^3)); du/dc = u through the mapped data
    sc = scenes.sphere_flow_scene(n_query=6)
    r = _run(sc, 2048)
    u, du = cf.sphere_flow(sc.query, sc.meta["a"])
    _check(r["u"], r["u_se"], u, 0.0, 3e-3)
    _check(r["du"], r["du_se"], du, 0.0, 3e-3)
    o = r["out"]
    dirichlet = np.nonzero(sc.neumann == 0)[0]
    hit = o["kind"][:, 0] == oracle.KIND_SHELL
    assert np.isin(o["elem"][hit], dirichlet).all()
    # no walk ends inside the sphere (the icosphere's inscribed radius bounds it)
    assert np.all(np.linalg.norm(o["x_end"], axis=1) >= 0.9 * sc.meta["a"])


def _on_neumann_points(name):
    """Query points on the Neumann part (off its vertices), with the scene."""
    if name == "quarter_disk":
        sc = scenes.quarter_disk_scene("mapped", n_query=2)
        s = (np.arange(6) + 0.37) / 16 + 0.1
        q = np.concatenate([np.stack([s, 0 * s], 1), np.stack([0 * s, s], 1)])
    elif name == "strip":
        sc = scenes.strip_scene(sigma=4.0, n_query=2)
        s = (np.arange(6) + 0.37) / 4 - 0.8
        q = np.concatenate([np.stack([s, np.full(6, -0.5)], 1), np.stack([s, np.full(6, 0.5)], 1)])
    else:
        sc = scenes.cube_neumann_scene(n_query=2)
        s = np.array([-0.63, -0.21, 0.17, 0.58])
        q = np.concatenate([np.stack([s, np.full(4, 1.0), 0.31 + 0 * s], 1),
                            np.stack([s, -0.27 + 0 * s, np.full(4, -1.0)], 1)])
    sc.query = q
    return sc


@pytest.mark.parametrize("name", ["quarter_disk", "strip", "cube"])
def test_query_points_on_the_neumann_part(name):
    # a query point on the Neumann part starts its walk there, with the element's normal
    # oriented out of the domain: the closed forms hold on that part too (u and du/dtheta;
    # du is a rare-event estimate near the fixed side, so its SE is floored at the median)
    sc = _on_neumann_points(name)
    r = _run(sc, 2048 if name == "cube" else 4096)
    if name == "quarter_disk":
        u, du = cf.quarter_disk(sc.query, "mapped")
        rel, ab, drel, dab = 3e-3, 2e-3, 0.08, 0.02
    elif name == "strip":
        u, du = cf.strip(sc.query, 4.0)
        rel, ab, drel, dab = 3e-3, 1e-3, 0.08, 0.01
    else:
        u, du = cf.cube_linear(sc.query)
        rel, ab, drel, dab = 0.0, 4e-3, 0.08, 0.02
    _check(r["u"], r["u_se"], u, rel, ab)
    _check(r["du"], np.maximum(r["du_se"], np.median(r["du_se"], axis=0)), du, drel, dab)
    # the first move goes into the domain (a normal pointing inwards would send it out)
    o = r["out"]
    assert np.all(np.isfinite(o["u_hat"]))
    x1 = o["x1"].reshape(-1, 3)
    x1 = x1[np.isfinite(x1[:, 0])]
    tol = 1e-12
    if name == "quarter_disk":
        assert np.all(x1[:, 0] >= -tol) and np.all(x1[:, 1] >= -tol)
        assert np.all(np.hypot(x1[:, 0], x1[:, 1]) <= 1 + tol)
    elif name == "strip":
        assert np.all(np.abs(x1[:, 1]) <= 0.5 + tol)
    else:
        assert np.all(np.abs(x1) <= 1 + tol)


def test_directions_at_an_edge_of_the_neumann_part():
    # A direction drawn on the Neumann part is turned into the domain.  On one side:
    # v -> -v where it points out (the inner half-sphere, uniform).  On an edge of two
    # sides: also mirrored into the wedge they bound; at a right angle that folds the
    # uniform sphere onto the uniform quarter-sphere (each fold is a symmetry of the
    # uniform distribution), so the moments are those of |v_i| with E|v_i| = 1/2 in 3D
    # (2/pi on the circle) and E v_i^2 = 1/d.
    rng = np.random.default_rng(7)
    n = 200_000
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    se = 4.0 / np.sqrt(n)
    one = oracle.turn_inward(v, [0.0, 0.0, 1.0])
    assert np.all(one[:, 2] <= 0)
    flip = v[:, 2] > 0
    assert np.array_equal(one[flip], -v[flip]) and np.array_equal(one[~flip], v[~flip])
    # the edge of the cube's faces y = -1 and z = 1 (outward normals -e_y, +e_z)
    q = oracle.turn_inward(v, [0.0, -1.0, 0.0], [0.0, 0.0, 1.0])
    assert np.all(q[:, 1] >= 0) and np.all(q[:, 2] <= 0)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(q.mean(0), [0.0, 0.5, -0.5], atol=se)
    np.testing.assert_allclose((q * q).mean(0), [1 / 3] * 3, atol=se)
    np.testing.assert_allclose((q[:, 0] * q[:, 1]).mean(), 0.0, atol=se)
    # the same edge with the sides the other way round: the same quarter-sphere
    q2 = oracle.turn_inward(v, [0.0, 0.0, 1.0], [0.0, -1.0, 0.0])
    assert np.all(q2[:, 1] >= 0) and np.all(q2[:, 2] <= 0)
    np.testing.assert_allclose(q2.mean(0), [0.0, 0.5, -0.5], atol=se)
    # a right-angled corner in 2D (the slab's corners): the uniform quarter-circle
    phi = rng.uniform(0, 2 * np.pi, n)
    c = np.stack([np.cos(phi), np.sin(phi), 0 * phi], 1)
    c2 = oracle.turn_inward(c, [1.0, 0.0, 0.0], [0.0, 1.0, 0.0])
    assert np.all(c2[:, :2] <= 0) and np.all(c2[:, 2] == 0)
    np.testing.assert_allclose(c2[:, :2].mean(0), [-2 / np.pi] * 2, atol=se)
    # a wedge of 60 degrees (y >= 0 and polar angle <= 60 deg): every direction ends inside
    a = np.pi / 3
    n_a = np.array([-np.sin(a), np.cos(a), 0.0])
    w = oracle.turn_inward(v, [0.0, -1.0, 0.0], n_a)
    assert np.all(w[:, 1] >= -1e-12) and np.all(w @ n_a <= 1e-12)


def test_ray_rules_on_the_slab():
    # The ray test against the Neumann part, on the thermal scene's slab (the box: elements 0-3,
    # the wire: 4-67, the slab polyline: 68-155; its underside y = 0.2 runs from x = -0.5 (68)
    # to 0.5 (107), then the right end x = 0.5 (108-111)).
    sc = scenes.thermal_scene(n_query=2)
    pr = to_oracle(sc)
    up = [0.0, 1.0]                       # the underside's normal out of the domain (into the slab)
    # a plain crossing from the domain below: the underside at t = 0.1
    t, e = oracle.ray_neumann(pr, [0.11, 0.1], [0.0, 1.0], 0.5)
    assert e == 92 and abs(t - 0.1) < 1e-12
    # a crossing up to 1e-5 tmax + 1e-4 eps past the ray's end counts, at the end
    t, e = oracle.ray_neumann(pr, [0.11, 0.1], [0.0, 1.0], 0.1 - 5e-7)
    assert e == 92 and t == 0.1 - 5e-7
    t, e = oracle.ray_neumann(pr, [0.11, 0.1], [0.0, 1.0], 0.1 - 1e-5)
    assert e == -1
    # a ray grazing the reflex corner (0.5, 0.2) from a walk on the last underside segment: the
    # end side lies behind the underside and is not hit, though the ray passes within the 1e-5
    # barycentric tolerance of its end (from a point not on the underside it is)
    v = [np.cos(1e-4), -np.sin(1e-4)]
    t, e = oracle.ray_neumann(pr, [0.4993, 0.2], v, 1e-3, skip=107, n_skip=up)
    assert e == -1 and t == 1e-3
    t, e = oracle.ray_neumann(pr, [0.4993, 0.2], v, 1e-3)
    assert e == 108
    # a ray nearly along the underside from a walk on it, rounding having put the walk 1e-8
    # inside the slab: the segments on its line are not hit (from the wrong side), adjacent or not
    x, v = [0.0125, 0.2 + 1e-8], [-1.0, -1e-7]
    t, e = oracle.ray_neumann(pr, x, v, 0.5, skip=88, n_skip=up)
    assert e == -1
    t, e = oracle.ray_neumann(pr, x, v, 0.5)
    assert e == 84
