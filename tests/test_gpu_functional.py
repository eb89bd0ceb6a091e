"""The volume-integrated functional on the GPU (dwos_sample_domain,
dwos_grad_l2_weighted, dwos_boundary_term_l2) against the oracle, and the
whole estimator against the screened disk's closed form."""
import numpy as np
import pytest

import oracle
from oracle import functional as fn
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle

pytestmark = pytest.mark.gpu


def torch_index(mask):
    import torch
    return torch.as_tensor(np.nonzero(mask)[0])


@pytest.fixture(scope="module")
def Solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300.dwos import Solver as S
    return S


@pytest.mark.parametrize("which", ["disk", "star", "sphere"])
def test_domain_samples_match_oracle(Solver, which):
    if which == "disk":
        sc, lo, hi = scenes.disk_scene("screened_1", n_query=4), [-1.1, -1.1], [1.1, 1.1]
    elif which == "star":
        sc, lo, hi = scenes.star_box_scene(n_seg=1024, n_query=4), [-0.6, -0.5], [0.7, 0.5]
    else:
        sc, lo, hi = scenes.sh_sphere_scene(freq=12, n_query=4), [-1.5, -1.5, -1.5], [1.5, 1.5, 1.5]
    s = Solver(0)
    s.load_scene(sc)
    pts, w = s.sample_domain(3000, lo, hi, seed=11)
    po, wo = fn.sample_domain(to_oracle(sc), 3000, lo, hi, seed=11)
    assert abs(w - wo) <= 1e-6 * wo
    p = pts.cpu().numpy()
    assert abs(len(p) - len(po)) <= 2          # a candidate within FP32 rounding of the boundary
    if len(p) == len(po):
        assert np.allclose(p, po, atol=2e-6)


@pytest.mark.parametrize("which", ["disk", "star", "sphere"])
def test_boundary_term_matches_oracle(Solver, which):
    if which == "disk":
        sc, lo, hi = scenes.disk_scene("mapped_cos", n_query=4), [-0.3, -2.0], [2.0, 2.0]
    elif which == "star":
        sc, lo, hi = scenes.star_box_scene(n_seg=1024, n_query=4), [-0.6, -0.6], [0.6, 0.6]
    else:
        sc, lo, hi = scenes.sh_sphere_scene(freq=12, n_query=4), [-1.5, -1.5, -1.5], [1.5, 1.5, 0.3]
    s = Solver(0)
    s.load_scene(sc)
    rng = np.random.default_rng(3)
    ur = rng.normal(size=len(sc.vert)) * 0.3
    g = s.boundary_term_l2(lo, hi, ur)
    go = fn.boundary_term_l2(to_oracle(sc), lo, hi, ur)
    assert np.allclose(g, go, rtol=1e-5, atol=1e-6 * np.abs(go).max()), np.abs(g - go).max()
    assert np.abs(go).max() > 0


def test_weighted_gradient_matches_oracle(Solver):
    sc = scenes.star_box_scene(n_seg=1024, n_query=4)
    s = Solver(0)
    s.load_scene(sc, K=2)
    pts, w = s.sample_domain(200, [-0.8, -0.8], [0.8, 0.8], seed=5)
    p = pts.cpu().numpy().astype(np.float64)
    # a sample inside the eps shell ends at once; FP32 and FP64 can disagree there and
    # each such walk carries a 1/h-amplified du/dn: compare on points off the shell
    far = oracle.closest_point(to_oracle(sc), p)[0] > 3 * sc.eps
    p = p[far]
    pts = pts[torch_index(far)]
    ur = (0.1 * p[:, 0]).astype(np.float32)
    wt = np.linspace(0.5, 1.5, len(p)).astype(np.float32) * w
    W = 64
    loss, g = (t.cpu().numpy() for t in s.grad_l2_weighted(pts, ur, wt, W))
    o = oracle.run_walks(to_oracle(sc, K=2), p.astype(np.float32).astype(np.float64), W, differential=True)
    go = fn.grad_l2_weighted(o["u_hat"], o["udot"], ur, wt, len(p), W, 8)
    lo_ = fn.loss_l2_weighted(o["u_hat"], ur, wt, len(p), W)
    # ~9k walks: a handful change branch between FP32 and FP64 (each with a 1/h-amplified
    # du/dn), so the comparison is at 1 % of the largest component; the weighting itself is
    # checked exactly below (a wrong weight moves the gradient by tens of percent)
    assert np.allclose(g, go, rtol=1e-2, atol=1e-2 * np.abs(go).max()), np.abs(g - go).max() / np.abs(go).max()
    assert abs(loss[0] - lo_) <= 1e-3 * abs(lo_) + 1e-8
    # the same walks: unit weights give dwos_grad_l2, constant weights scale it
    g1 = s.grad_l2_weighted(pts, ur, np.ones(len(p), np.float32), W)[1].cpu().numpy()
    g0 = s.grad_l2(pts, ur, W)[1].cpu().numpy()
    g2 = s.grad_l2_weighted(pts, ur, np.full(len(p), 2.5, np.float32), W)[1].cpu().numpy()
    assert np.allclose(g1, g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())
    assert np.allclose(g2, 2.5 * g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())


def test_functional_gradient_matches_the_closed_form(Solver):
    from scipy.integrate import quad
    from scipy.special import iv
    J = lambda R: quad(lambda r: 0.5 * (iv(0, 2 * r) / iv(0, 2 * R)) ** 2 * 2 * np.pi * r, 0, R, epsabs=1e-13)[0]
    want = (J(1 + 1e-5) - J(1 - 1e-5)) / 2e-5
    sc = scenes.disk_scene("screened_1", n_query=4)
    s = Solver(0)
    s.load_scene(sc)
    vals = []
    for rep in range(6):
        Jv, g = s.functional_gradient([-1, -1], [1, 1], lambda x: np.zeros(len(x)), walks=256, n_try=8192,
                                      seed=rep + 1, walk_id_base=rep << 36)
        vals.append(g[0])
    vals = np.array(vals)
    se = vals.std(ddof=1) / np.sqrt(len(vals))
    print("dJ/dR: estimate %.4f +- %.4f, closed form %.4f" % (vals.mean(), se, want))
    # boundary part pi (exact); the domain part carries the eps/h bias of the du/dn estimate
    # (Sec. 5.3; 4.4 % low at eps/h = 0.1 in the oracle): budget 6 % of it
    assert abs(vals.mean() - want) < 4.5 * se + 0.06 * abs(want - np.pi)
