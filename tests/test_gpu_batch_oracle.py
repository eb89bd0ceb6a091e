"""The batched launch (one persistent walk launch per dimension over a table of
problem descriptors in shared memory, lanes refilled across problems) against
the FP64 oracle, walk by walk and job by job.

The batch mixes 2D star-in-box and 3D SH-sphere-in-box problems at the corners
of the batched workload's ranges: sigma = 0.01 and 100, and one 200,000-triangle
mesh.  Each job's records and traces from one pass are replayed by walk id in
the oracle (walk id = the job's base + p W + w); on walks whose branch matches,
u and udot agree to the per-walk bounds of the single-problem parity tests, and
each job's U-statistic gradient and loss agree with the oracle's estimators on
the same walks.
"""
import numpy as np
import pytest

import oracle
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle
from tests.test_gpu_parity import check_walks, gpu_udot

pytestmark = pytest.mark.gpu


def _problems():
    out = [
        scenes.star_box_scene(n_seg=2000, n_modes=8, sigma=0.01, n_query=6, walks=32, seed=101),
        scenes.star_box_scene(n_seg=6000, n_modes=8, sigma=100.0, n_query=6, walks=32, seed=102),
        scenes.sh_sphere_scene(freq=100, lmax=3, coef_std=0.02, sigma=0.01, n_query=4, walks=16, seed=103),
        scenes.sh_sphere_scene(freq=16, lmax=3, coef_std=0.02, sigma=100.0, n_query=6, walks=32, seed=104),
        scenes.sh_sphere_scene(freq=30, lmax=3, coef_std=0.02, sigma=1.0, n_query=6, walks=32, seed=105),
    ]
    for sc in out:
        if sc.u_ref is None:
            sc.u_ref = np.full(sc.query.shape[0], 0.1)
    return out


@pytest.fixture(scope="module")
def batch_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    probs = _problems()
    assert max(len(sc.elem) for sc in probs) >= 200_000
    solvers = []
    for sc in probs:
        s = dwos.Solver(0)
        s.load_scene(sc)
        solvers.append(s)
    bases = [(7 + i) << 36 for i in range(len(probs))]
    b = dwos.Batch([(s, sc.query, sc.walks, sc.u_ref, base) for sc, s, base in zip(probs, solvers, bases)])
    b.trace(True)
    b.run()
    res = b.results()
    recs = [b.records(i, trace=True) for i in range(len(probs))]
    st = b.stats()
    return probs, bases, res, recs, st


def test_batched_walks_replay_in_the_oracle(batch_run):
    probs, bases, res, recs, st = batch_run
    assert st["capped"] == 0
    for i, (sc, base) in enumerate(zip(probs, bases)):
        rec, tr = recs[i]
        o = oracle.run_walks(to_oracle(sc), sc.query, sc.walks, differential=True, walk_id_base=base)
        same = check_walks(sc, {"rec": rec, "trace": tr}, o, max_flip=0.03)
        print("%s (%d elements, sigma %.3g): %.4f of walks on the same branch"
              % (sc.name, len(sc.elem), sc.sigma, same.mean()))
        # job sums: the oracle's estimators on the same walks; a walk whose branch changed
        # (counted above, rare) enters with the GPU's own values, so that the comparison
        # tests the batch's reductions rather than the FP32/FP64 branch flip
        n = sc.query.shape[0]
        u_w = np.where(same, o["u_hat"], rec["u"].astype(np.float64))
        ud_w = np.where(same[:, None], o["udot"], gpu_udot(sc, rec))
        go = est.grad_l2_ustat(u_w, ud_w, sc.u_ref, n, sc.walks, sc.B)
        lo = est.loss_l2(u_w, sc.u_ref, n, sc.walks)
        g = res[i]["grad"]
        scale = np.abs(go).max()
        assert np.allclose(g, go, rtol=2e-3, atol=2e-3 * scale), (i, np.abs(g - go).max() / scale)
        assert abs(res[i]["loss"] - lo) <= 1e-4 * abs(lo) + 1e-7
        assert np.allclose(res[i]["u_mean"], u_w.reshape(n, sc.walks).mean(1), rtol=1e-4, atol=1e-6)
