"""Pins for the oracle's brute-force DistanceToBoundary and inside test."""
import numpy as np

import oracle
from paper_2405_12964_gb300 import scenes


def _prob(vert, elem):
    return oracle.Problem(vert=np.asarray(vert, float), elem=np.asarray(elem, np.int32),
                          data_kind="mapped", g_vert=np.zeros(len(vert)))


def test_segment_closest_point_matches_dense_sampling():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.normal(size=2), rng.normal(size=2)
        pr = _prob([a, b], [[0, 1]])
        p = rng.normal(size=(8, 2)) * 2
        d, xb, e, bary = oracle.closest_point(pr, p)
        t = np.linspace(0, 1, 20001)
        seg = a[None] + t[:, None] * (b - a)[None]
        dd = np.linalg.norm(p[:, None, :] - seg[None], axis=2)
        assert np.allclose(d, dd.min(axis=1), atol=2e-4 * np.linalg.norm(b - a))
        assert np.allclose(xb, a + bary[:, :1] * (b - a), atol=1e-12)
        assert np.allclose(np.linalg.norm(p - xb, axis=1), d, atol=1e-12)


def test_triangle_closest_point_matches_dense_barycentric_grid():
    rng = np.random.default_rng(2)
    n = 400
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    m = (i + j) <= n
    w1, w2 = (i[m] / n), (j[m] / n)
    for _ in range(12):
        A, B, C = rng.normal(size=(3, 3))
        pr = _prob([A, B, C], [[0, 1, 2]])
        p = rng.normal(size=(6, 3)) * 1.5
        d, xb, e, bary = oracle.closest_point(pr, p)
        pts = A[None] + w1[:, None] * (B - A)[None] + w2[:, None] * (C - A)[None]
        dd = np.linalg.norm(p[:, None, :] - pts[None], axis=2).min(axis=1)
        h = max(np.linalg.norm(B - A), np.linalg.norm(C - A)) / n
        assert np.all(d <= dd + 1e-12)            # never farther than any sampled point
        assert np.all(dd - d <= 2 * h)             # and within the grid resolution
        recon = A + bary[:, :1] * (B - A) + bary[:, 1:2] * (C - A)
        assert np.allclose(recon, xb, atol=1e-12)
        assert np.all(bary >= -1e-12) and np.all(bary.sum(1) <= 1 + 1e-12)


def test_triangle_face_region_is_orthogonal_projection():
    A, B, C = np.array([0., 0, 0]), np.array([1., 0, 0]), np.array([0., 1, 0])
    pr = _prob([A, B, C], [[0, 1, 2]])
    p = np.array([[0.2, 0.3, 0.7], [0.25, 0.25, -2.0]])
    d, xb, e, bary = oracle.closest_point(pr, p)
    assert np.allclose(d, [0.7, 2.0])
    assert np.allclose(xb, [[0.2, 0.3, 0], [0.25, 0.25, 0]])
    assert np.allclose(bary, [[0.2, 0.3], [0.25, 0.25]])


def test_tie_break_prefers_smallest_element_index():
    v = [[0., 0.], [1., 0.]]
    pr = _prob(v, [[0, 1], [1, 0], [0, 1]])
    d, xb, e, bary = oracle.closest_point(pr, np.array([[0.5, 0.5]]))
    assert e[0] == 0


def test_brute_force_matches_analytic_disk_distance():
    sc = scenes.disk_scene("screened_1")
    pr = _prob(sc.vert, sc.elem)
    d, xb, e, bary = oracle.closest_point(pr, sc.query)
    r = np.linalg.norm(sc.query, axis=1)
    sag = 1 - np.cos(np.pi / 128)
    assert np.all(d <= 1 - r + 1e-12) and np.all(d >= 1 - r - sag)


def test_inside_parity_disk_box_star_and_sphere():
    sc = scenes.disk_scene("screened_1")
    pr = _prob(sc.vert, sc.elem)
    rng = np.random.default_rng(3)
    p = rng.uniform(-1.3, 1.3, size=(400, 2))
    r = np.linalg.norm(p, axis=1)
    keep = np.abs(r - 1) > 0.01
    assert np.array_equal(oracle.inside(pr, p[keep]), r[keep] < 1)
    st = scenes.star_box_scene(n_seg=256)
    pr = _prob(st.vert, st.elem)
    p = rng.uniform(-0.95, 0.95, size=(400, 2))
    rr = np.linalg.norm(p, axis=1)
    keep = (rr > 0.45) | (rr < 0.15)
    assert np.array_equal(oracle.inside(pr, p[keep]), rr[keep] > 0.45)   # in box, outside star
    v, f = scenes.icosphere(4)
    pr = _prob(v, f)
    p = rng.uniform(-1.2, 1.2, size=(300, 3))
    r = np.linalg.norm(p, axis=1)
    keep = (r < 0.9) | (r > 1.01)
    assert np.array_equal(oracle.inside(pr, p[keep]), r[keep] < 0.9)
