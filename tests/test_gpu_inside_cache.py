"""The inside flags a call keeps for the next one.

A walk-running call tests its query points against Omega (ray parity) and
keeps the flags with the points; the next call reuses the flag of every point
equal to its stored copy bit for bit, and tests the others.  A new geometry
(set_boundary, set_params, set_neumann) drops the stored flags.  These tests
move points in and out of Omega between calls and check every point's flag
through the records: a point outside gets NaN records (and DWOS_ERR_OUTSIDE),
a point inside finite ones, whatever the previous calls were.
"""
import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300.dwos import DwosError, Solver
    return torch, Solver, DwosError


def test_flags_follow_points_and_geometry(env):
    torch, Solver, DwosError = env
    sc = scenes.translated_star_scene(n_seg=1024, n_query=8)
    s = Solver(0)
    s.load_scene(sc)
    s.set_boundary(sc.reference_vertices(), sc.elem, sc.jac)
    s.set_dirichlet_mapped(sc.g_vert)
    rng = np.random.default_rng(8)
    pts = rng.uniform(-0.9, 0.9, size=(256, 2)).astype(np.float32)
    want = s.inside(pts).cpu().numpy().astype(bool)
    assert want.any() and (~want).any()

    # the flags as the walks saw them: dwos_eval on device memory gives a NaN mean for a
    # point outside Omega (reported as DWOS_ERR_OUTSIDE by the next sync)
    def ran(p):
        out = s.eval(torch.as_tensor(p, device="cuda"), 8)
        m = out["u"].cpu().numpy()
        try:
            s.sync()
        except DwosError as e:
            assert e.status == 8
        return np.isfinite(m)

    assert np.array_equal(ran(pts), want)            # first call: every flag computed
    assert np.array_equal(ran(pts), want)            # same points: flags reused
    # move a few points across the boundary (in and out of the star) and back
    p2 = pts.copy()
    flip = rng.choice(len(pts), 40, replace=False)
    p2[flip] = np.where(want[flip, None], np.float32(0.0), np.float32(0.85))   # star centre is outside Omega
    want2 = s.inside(p2).cpu().numpy().astype(bool)
    assert not np.array_equal(want2, want)
    assert np.array_equal(ran(p2), want2)
    assert np.array_equal(ran(pts), want)
    # one coordinate changed by one ulp still counts as a new point (and is tested again)
    p3 = pts.copy()
    p3[:, 0] = np.nextafter(p3[:, 0], np.float32(2.0))
    assert np.array_equal(ran(p3), s.inside(p3).cpu().numpy().astype(bool))
    # a different point count drops the stored flags
    assert np.array_equal(ran(pts[:100]), want[:100])
    assert np.array_equal(ran(pts), want)
    # a new geometry drops them: move the star by a refit, then by a rebuild
    for theta in (np.array([0.3, 0.0]), np.array([-0.25, 0.2])):
        s.set_params(theta)
        wt = s.inside(pts).cpu().numpy().astype(bool)
        assert not np.array_equal(wt, want)
        assert np.array_equal(ran(pts), wt)
    s.set_boundary(sc.reference_vertices(), sc.elem, sc.jac)
    s.set_dirichlet_mapped(sc.g_vert)
    assert np.array_equal(ran(pts), want)
