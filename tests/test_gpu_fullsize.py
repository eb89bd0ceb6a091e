"""Parity at full size, in the launch configuration bench.py times: run every
walk of the 2D shape-from-diffusion workload (256 x 4096) and of the 3D thermal
workload (200k triangles, 4096 x 2048), then replay sampled walks in the oracle
by their walk ids and compare them one by one."""
import numpy as np
import pytest

import oracle
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle
from tests.test_gpu_parity import branch_match, gpu_udot

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


def _sampled_parity(Solver, sc, n_pts, per_pt, max_flip):
    s = Solver(0)
    s.load_scene(sc)
    W = sc.walks
    g = s.walk_records(sc.query, W, trace=True)
    st = s.stats()
    assert st["capped"] == 0
    rng = np.random.default_rng(11)
    pts = rng.choice(sc.query.shape[0], size=n_pts, replace=False)
    same_all, n = 0, 0
    for p in pts:
        w0 = int(rng.integers(0, W - per_pt))
        rows = slice(p * W + w0, p * W + w0 + per_pt)
        o = oracle.run_walks(to_oracle(sc), sc.query[p:p + 1], per_pt, differential=True,
                             walk_id_base=p * W + w0)
        gg = {"rec": g["rec"][rows], "trace": g["trace"][rows]}
        same = branch_match(sc, gg, o)
        ug = gg["rec"]["u"].astype(np.float64)
        assert np.all(np.abs(ug - o["u_hat"])[same] <= 1e-4 * np.abs(o["u_hat"][same]) + 1e-5)
        dg = gpu_udot(sc, gg["rec"])
        assert np.all(np.abs(dg - o["udot"])[same] <= 1e-3 * (1 + np.abs(o["udot"][same])))
        same_all += same.sum()
        n += per_pt
    assert 1 - same_all / n <= max_flip


def test_fullsize_star_box_sampled_walks(Solver):
    _sampled_parity(Solver, scenes.star_box_scene(), n_pts=16, per_pt=16, max_flip=0.02)


def test_fullsize_thermal_3d_sampled_walks(Solver):
    _sampled_parity(Solver, scenes.sh_sphere_scene(), n_pts=6, per_pt=8, max_flip=0.05)
