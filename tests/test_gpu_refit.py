"""Parameter updates refit the BVH instead of rebuilding it.

dwos_set_params moves the vertices and refits the boxes over the tree it
has (no host synchronisation).  The searches are exact, so a refit tree and
a tree built afresh for the same vertices give the same closest distances
bit for bit and the same closest elements but for ties between equally
distant elements, and the same walks.  Search order 1 (Morton-cell climb)
needs a fresh tree: while it is selected, updates rebuild.
"""
import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300.dwos import Solver as S
    return S


def _pair(Solver, sc, path, traversal):
    """A: reference vertices, then theta along `path` (refits); B: built at the last theta."""
    a = Solver(0)
    a.load_scene(sc, traversal=traversal)
    a.set_boundary(sc.reference_vertices(), sc.elem, sc.jac)
    a.set_dirichlet_mapped(sc.g_vert)
    for th in path:
        a.set_params(th)
    b = Solver(0)
    b.load_scene(sc, traversal=traversal)
    # the vertices the device forms, v_ref + 1 * theta rounded once in FP32 (the star's
    # Jacobian is the identity, the box's zero)
    v = sc.reference_vertices().astype(np.float32)
    v[4:] = v[4:] + np.asarray(path[-1], dtype=np.float32)
    b.set_boundary(v, sc.elem, None)
    b.set_dirichlet_mapped(sc.g_vert)
    return a, b


@pytest.mark.parametrize("traversal", [0, 3])
def test_refit_tree_gives_the_fresh_tree_results(Solver, traversal):
    sc = scenes.translated_star_scene(n_seg=1024, n_query=32)
    sc.walks = 256
    path = [np.array([0.004 * i, -0.0026 * i]) for i in range(1, 40)]   # 39 refits
    a, b = _pair(Solver, sc, path, traversal)
    rng = np.random.default_rng(5)
    p = rng.uniform(-0.95, 0.95, size=(20000, 2))
    da, ea, _ = (t.cpu().numpy() for t in a.closest_point(p))
    db, eb, _ = (t.cpu().numpy() for t in b.closest_point(p))
    assert np.array_equal(da, db)
    assert (ea == eb).mean() > 0.999
    ra = a.walk_records(sc.query, sc.walks, walk_id_base=11)["rec"]
    rb = b.walk_records(sc.query, sc.walks, walk_id_base=11)["rec"]
    assert np.array_equal(ra["u"], rb["u"]) and np.array_equal(ra["meta"], rb["meta"])
    assert (ra["elem"] == rb["elem"]).mean() > 0.999
    # the refit tree's boxes still hold every element: nothing beyond the tree's size
    a.sync()


def test_order_1_after_refits_and_periodic_rebuild(Solver):
    sc = scenes.translated_star_scene(n_seg=1024, n_query=16)
    path = [np.array([0.001 * i, 0.002 * i]) for i in range(1, 70)]  # past the rebuild every 64 updates
    a, b = _pair(Solver, sc, path, 1)
    rng = np.random.default_rng(6)
    p = rng.uniform(-0.95, 0.95, size=(5000, 2))
    da, _, _ = (t.cpu().numpy() for t in a.closest_point(p))
    db, _, _ = (t.cpu().numpy() for t in b.closest_point(p))
    assert np.array_equal(da, db)
    # switching a refit context to order 1 runs it as order 0 until the next rebuild
    c, d = _pair(Solver, sc, path[:5], 3)
    c.set_options(traversal=1)
    dc, _, _ = (t.cpu().numpy() for t in c.closest_point(p))
    dd, _, _ = (t.cpu().numpy() for t in d.closest_point(p))
    assert np.array_equal(dc, dd)
