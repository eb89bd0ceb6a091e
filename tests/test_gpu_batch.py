"""Batched problems (one walk launch per dimension over a table of problems,
then per-problem reductions; optionally one captured CUDA graph): the results
equal those of separate dwos_grad_l2 calls on the same walks."""
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
    from paper_2405_12964_gb300 import dwos
    probs = scenes.batched_problems(n=8, scale=0.05, max_elems=20000, seed=7)
    solvers = []
    for sc in probs:
        s = dwos.Solver(0)
        s.load_scene(sc)
        solvers.append(s)
    return torch, dwos, probs, solvers


def _separate(torch, probs, solvers):
    out = []
    for sc, s in zip(probs, solvers):
        loss, g = s.grad_l2(sc.query, sc.u_ref, sc.walks, walk_id_base=1000)
        torch.cuda.synchronize()
        out.append((float(loss[0]), g.cpu().numpy()))
    return out


def _compare(res, ref):
    for r, (loss, g) in zip(res, ref):
        assert abs(r["loss"] - loss) <= 1e-9 * max(1.0, abs(loss))
        assert np.allclose(r["grad"], g, rtol=1e-7, atol=1e-10 * max(1.0, np.abs(g).max()))


def test_batch_pass_equals_separate_calls(env):
    torch, dwos, probs, solvers = env
    assert {sc.dim for sc in probs} == {2, 3}
    ref = _separate(torch, probs, solvers)
    b = dwos.Batch([(s, sc.query, sc.walks, sc.u_ref, 1000) for sc, s in zip(probs, solvers)])
    b.run()
    _compare(b.results(), ref)
    st = b.stats()
    assert st["walks"] == sum(sc.query.shape[0] * sc.walks for sc in probs)
    assert st["capped"] == 0


def test_batch_graph_replay_and_autotune(env):
    torch, dwos, probs, solvers = env
    ref = _separate(torch, probs, solvers)
    b = dwos.Batch([(s, sc.query, sc.walks, sc.u_ref, 1000) for sc, s in zip(probs, solvers)])
    b.capture()
    for _ in range(2):
        b.launch()
        _compare(b.results(), ref)
    b.autotune(reps=1)
    for dim in (2, 3):
        cfg = b.config(dim)
        assert cfg["block_size"] in (128, 256) and cfg["blocks_per_sm"] >= 1 and cfg["traversal"] in (0, 1, 2, 3)
    b.launch()
    _compare(b.results(), ref)
