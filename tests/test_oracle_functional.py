"""The volume-integrated functional (Eqs. functional, functional_deriv) in the
oracle.

Pins:
  * the monomial integrals against dense quadrature on random segments and
    triangles (the boundary term's integration);
  * the boundary term on the disk: V_n = 1 for the radius, so with g = 1 it is
    half the polygon's perimeter; a Fourier mode integrates to about zero;
  * the sampled domain's weight x count estimates the disk's area;
  * the whole estimator's mean equals dJ/dR of J(R) = int_disk 1/2 u^2 for the
    screened disk u = I0(k r) / I0(k R), computed by quadrature, within its
    standard error and the estimator's eps/h bias (Sec. 5.3): the domain term
    comes out 4.4 % low at eps/h = 0.1 (2.8 % with eps and h four times
    smaller, 14 % at eps/h = 0.4), so the budget is 6 % of the domain term.
"""
import numpy as np
import pytest

import oracle
from oracle import functional as fn
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle


def test_monomial_integrals_match_dense_quadrature():
    rng = np.random.default_rng(0)
    # segment of length L: midpoint rule with many points
    L = 1.7
    t = (np.arange(20000) + 0.5) / 20000
    for exps in [(1, 2), (3, 0), (2, 2)]:
        want = L * np.mean((1 - t) ** exps[0] * t ** exps[1])
        assert abs(fn._simplex_monomial(L, list(exps)) - want) < 1e-7
    # triangle of area A: uniform samples of the barycentrics (large count, Monte Carlo)
    A = 0.8
    u = rng.random((400000, 2))
    flip = u.sum(1) > 1
    u[flip] = 1 - u[flip]
    w = np.stack([1 - u.sum(1), u[:, 0], u[:, 1]], 1)
    for exps in [(1, 1, 1), (2, 1, 0), (0, 0, 3)]:
        vals = A * np.prod(w ** np.array(exps), axis=1)
        want, se = vals.mean(), vals.std() / np.sqrt(len(vals))
        assert abs(fn._simplex_monomial(A, list(exps)) - want) < 5 * se


def test_boundary_term_on_the_disk():
    sc = scenes.disk_scene("screened_1", n_query=4)
    pr = to_oracle(sc)
    g = fn.boundary_term_l2(pr, [-2, -2], [2, 2])
    n = len(sc.elem)
    perimeter = 2 * n * np.sin(np.pi / n)
    # dJ/dR of the boundary part: int 1/2 g^2 V_n dA with V_n = the radial unit ... on a polygon the
    # vertices move radially, so V_n = cos(pi/n) along each edge
    assert abs(g[0] - 0.5 * perimeter * np.cos(np.pi / n)) < 1e-12
    assert np.all(np.abs(g[1:]) < 1e-12)
    # a mask box that excludes every element
    assert np.all(fn.boundary_term_l2(pr, [-0.5, -0.5], [0.5, 0.5]) == 0)


def test_domain_weights_estimate_the_area():
    sc = scenes.disk_scene("screened_1", n_query=4)
    pr = to_oracle(sc)
    pts, w = fn.sample_domain(pr, 4000, [-1.1, -1.1], [1.1, 1.1], seed=7)
    n = len(sc.elem)
    area = 0.5 * n * np.sin(2 * np.pi / n)
    p = area / 2.2 ** 2
    se = 2.2 ** 2 * np.sqrt(p * (1 - p) / 4000)
    assert abs(len(pts) * w - area) < 4.5 * se
    assert np.all(np.hypot(pts[:, 0], pts[:, 1]) < 1.0)


def _disk_J(R, k=2.0):
    from scipy.integrate import quad
    from scipy.special import iv
    return quad(lambda r: 0.5 * (iv(0, k * r) / iv(0, k * R)) ** 2 * 2 * np.pi * r, 0, R, epsabs=1e-13)[0]


def test_estimator_mean_matches_the_closed_form():
    sc = scenes.disk_scene("screened_1", n_query=4)
    pr = to_oracle(sc)
    want = (_disk_J(1 + 1e-5) - _disk_J(1 - 1e-5)) / 2e-5
    est_g = []
    for rep in range(8):
        pts, w = fn.sample_domain(pr, 1500, [-1, -1], [1, 1], seed=100 + rep)
        W = 64
        o = oracle.run_walks(pr, pts, W, differential=True, walk_id_base=rep << 32)
        ur = np.zeros(len(pts))
        est_g.append(fn.grad_l2_weighted(o["u_hat"], o["udot"], ur, np.full(len(pts), w), len(pts), W, 8)[0])
    gb = fn.boundary_term_l2(pr, [-1.5, -1.5], [1.5, 1.5])[0]
    # the boundary term is exact here: pi (g = 1, V_n = 1 on the unit circle, to the polygon's sagitta)
    assert abs(gb - np.pi) < 2e-3
    tot = np.array(est_g) + gb
    se = tot.std(ddof=1) / np.sqrt(len(tot))
    assert abs(tot.mean() - want) < 4.5 * se + 0.06 * abs(want - gb), (tot.mean(), want, se)


# ---- boundary loss of the general functional (App. C) ----------------------

def _perturbed(pr, sc, delta):
    """The oracle problem at theta = delta (vertices v + J delta, data g + dg delta)."""
    v = np.asarray(sc.vert, dtype=np.float64) + np.einsum("vkp,p->vk", np.asarray(sc.jac, dtype=np.float64), delta)
    g = np.asarray(sc.g_vert, dtype=np.float64)
    if sc.dg_vert is not None:
        g = g + np.asarray(sc.dg_vert, dtype=np.float64) @ delta
    return to_oracle(sc, vert=v, g_vert=g)


def test_boundary_loss_on_the_polygon():
    # g = 1 on a regular 128-gon of radius R: J_b = 1/2 perimeter = 128 R sin(pi/128), linear in R;
    # the Fourier modes change the perimeter only at second order
    sc = scenes.disk_scene("screened_1", n_query=4)
    pr = to_oracle(sc)
    n = len(sc.elem)
    loss, g = fn.boundary_loss_l2(pr, [-2, -2], [2, 2])
    assert abs(loss - n * np.sin(np.pi / n)) < 1e-12
    assert abs(g[0] - n * np.sin(np.pi / n)) < 1e-12
    assert np.all(np.abs(g[1:]) < 1e-12)
    # a target equal to the data gives zero; a mask box around no element gives zero
    ub = np.asarray(sc.g_vert, dtype=np.float64)
    l0, g0 = fn.boundary_loss_l2(pr, [-2, -2], [2, 2], ub)
    assert l0 == 0.0 and np.all(g0 == 0.0)
    lm, gm = fn.boundary_loss_l2(pr, [-0.5, -0.5], [0.5, 0.5])
    assert lm == 0.0 and np.all(gm == 0.0)
    # the right half-plane box keeps the elements whose centres have x >= 0: half of them
    lh, _ = fn.boundary_loss_l2(pr, [0.0, -2], [2, 2])
    assert abs(lh - 0.5 * loss) < 1e-12


def test_boundary_loss_on_the_sphere():
    # unperturbed SH sphere (radius 1) with g = 1, target 0, mask around the sphere only:
    # J_b = A / 2 with A the mesh's area; the l = 0 coefficient moves every sphere vertex by
    # Y00 along its radius, and A scales as R^2, so dJ_b/dc00 = A Y00
    sc = scenes.sh_sphere_scene(freq=6, n_query=4, coeffs=np.zeros(81))
    pr = to_oracle(sc)
    loss, g = fn.boundary_loss_l2(pr, [-1.5] * 3, [1.5] * 3)
    vert, elem = np.asarray(sc.vert, dtype=np.float64), np.asarray(sc.elem)
    sph = np.all(np.abs(vert[elem].mean(axis=1)) <= 1.5, axis=1)
    tri = vert[elem[sph]]
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    y00 = 0.5 / np.sqrt(np.pi)
    assert abs(loss - 0.5 * area) < 1e-12 * area
    assert abs(g[0] - area * y00) < 1e-10 * area


def test_boundary_loss_gradient_matches_central_differences():
    # a small star in its box, random per-vertex data with a data derivative, a random target
    # and a mask that cuts through both the star and the box: the gradient equals central
    # differences of the value (a separate formula: no derivative code involved)
    rng = np.random.default_rng(5)
    sc = scenes.star_box_scene(n_seg=96, n_query=4)
    nv, N = len(sc.vert), sc.jac.shape[2]
    sc.g_vert = rng.uniform(0.0, 1.0, nv)
    sc.dg_vert = rng.normal(0.0, 0.3, (nv, N))
    ub = rng.uniform(0.0, 1.0, nv)
    lo, hi = [-0.9, -1.2], [1.2, 0.25]
    pr = _perturbed(None, sc, np.zeros(N))
    loss, g = fn.boundary_loss_l2(pr, lo, hi, ub)
    assert abs(loss - fn.boundary_loss_l2_value(pr, lo, hi, ub)) < 1e-14
    h = 1e-6
    fd = np.zeros(N)
    for j in range(N):
        e = np.zeros(N)
        e[j] = h
        fd[j] = (fn.boundary_loss_l2_value(_perturbed(None, sc, e), lo, hi, ub)
                 - fn.boundary_loss_l2_value(_perturbed(None, sc, -e), lo, hi, ub)) / (2 * h)
    assert np.abs(g).max() > 1e-3
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())


def test_boundary_loss_gradient_matches_central_differences_3d():
    rng = np.random.default_rng(6)
    sc = scenes.sh_sphere_scene(freq=4, lmax=3, n_query=4)
    nv, N = len(sc.vert), sc.jac.shape[2]
    sc.g_vert = rng.uniform(0.0, 1.0, nv)
    sc.dg_vert = rng.normal(0.0, 0.3, (nv, N))
    ub = rng.uniform(0.0, 1.0, nv)
    lo, hi = [-2.5, -0.3, -2.5], [0.4, 2.5, 2.5]
    pr = _perturbed(None, sc, np.zeros(N))
    loss, g = fn.boundary_loss_l2(pr, lo, hi, ub)
    h = 1e-6
    fd = np.zeros(N)
    for j in range(N):
        e = np.zeros(N)
        e[j] = h
        fd[j] = (fn.boundary_loss_l2_value(_perturbed(None, sc, e), lo, hi, ub)
                 - fn.boundary_loss_l2_value(_perturbed(None, sc, -e), lo, hi, ub)) / (2 * h)
    assert np.abs(g).max() > 1e-3
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())
