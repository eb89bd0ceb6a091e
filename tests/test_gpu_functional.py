"""The volume-integrated functional on the GPU (dwos_sample_domain,
dwos_grad_l2_weighted, dwos_boundary_term_l2) against the oracle, and the
whole estimator against the screened disk's closed form."""
import numpy as np
import pytest

import oracle
from oracle import functional as fn
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle
from tests.test_gpu_parity import branch_match, gpu_udot

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
    # ~9k walks: a handful change branch between FP32 and FP64, each with a 1/h-amplified
    # du/dn.  As in the per-walk tests, those walks are identified by their branch (steps and
    # termination per phase, terminal element) and enter the oracle's estimator with the
    # GPU's own per-walk values; every other walk is the oracle's
    rec = s.walk_records(pts, W, trace=True)
    same = branch_match(sc, rec, o)
    assert same.mean() >= 0.99, same.mean()
    u_w = np.where(same, o["u_hat"], rec["rec"]["u"].astype(np.float64))
    ud_w = np.where(same[:, None], o["udot"], gpu_udot(sc, rec["rec"]))
    go = fn.grad_l2_weighted(u_w, ud_w, ur, wt, len(p), W, 8)
    lo_ = fn.loss_l2_weighted(u_w, ur, wt, len(p), W)
    assert np.allclose(g, go, rtol=3e-3, atol=3e-3 * np.abs(go).max()), np.abs(g - go).max() / np.abs(go).max()
    assert abs(loss[0] - lo_) <= 1e-4 * abs(lo_) + 1e-8
    # the same walks: unit weights give dwos_grad_l2, constant weights scale it
    g1 = s.grad_l2_weighted(pts, ur, np.ones(len(p), np.float32), W)[1].cpu().numpy()
    g0 = s.grad_l2(pts, ur, W)[1].cpu().numpy()
    g2 = s.grad_l2_weighted(pts, ur, np.full(len(p), 2.5, np.float32), W)[1].cpu().numpy()
    assert np.allclose(g1, g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())
    # the per-walk weights are FP32: a factor of 2.5 rounds each walk's term afresh
    # (relative 2^-24 a term), the FP64 sums over walks then differ in the last FP32 bits
    assert np.allclose(g2, 2.5 * g0, rtol=1e-6, atol=1e-6 * np.abs(g0).max())


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


def _f32(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("which", ["star", "sphere"])
def test_boundary_loss_matches_oracle(Solver, which):
    # App. C's boundary loss, exact on both sides: the GPU (FP64 from the FP32 inputs) against
    # the oracle on the same FP32-rounded vertices, Jacobian, data, data derivative and target
    rng = np.random.default_rng(11)
    if which == "star":
        sc, lo, hi = scenes.star_box_scene(n_seg=1024, n_query=4), [-0.83, -1.31], [1.27, 0.217]
    else:
        sc, lo, hi = scenes.sh_sphere_scene(freq=12, lmax=4, n_query=4), [-2.5, -0.31, -2.5], [0.43, 2.5, 2.5]
    nv, N = len(sc.vert), sc.jac.shape[2]
    sc.g_vert = rng.uniform(0.0, 1.0, nv)
    sc.dg_vert = rng.normal(0.0, 0.3, (nv, N))
    ub = rng.uniform(0.0, 1.0, nv).astype(np.float32)
    s = Solver(0)
    s.load_scene(sc)
    loss, g = s.boundary_loss_l2(lo, hi, ub)
    pr = to_oracle(sc, vert=_f32(sc.vert), jac=_f32(sc.jac), g_vert=_f32(sc.g_vert), dg_vert=_f32(sc.dg_vert))
    want_loss, want_g = fn.boundary_loss_l2(pr, lo, hi, ub.astype(np.float64))
    assert want_loss > 0 and np.abs(want_g).max() > 0
    assert abs(loss - want_loss) <= 1e-9 * want_loss
    assert np.allclose(g, want_g, rtol=1e-8, atol=1e-10 * np.abs(want_g).max())
    # without a target and without a data derivative
    s.set_dirichlet_mapped(sc.g_vert)
    loss0, g0 = s.boundary_loss_l2(lo, hi)
    pr0 = to_oracle(sc, vert=_f32(sc.vert), jac=_f32(sc.jac), g_vert=_f32(sc.g_vert), dg_vert=None)
    wl0, wg0 = fn.boundary_loss_l2(pr0, lo, hi)
    assert abs(loss0 - wl0) <= 1e-9 * wl0
    assert np.allclose(g0, wg0, rtol=1e-8, atol=1e-10 * np.abs(wg0).max())


def test_boundary_loss_rejects_field_data_and_bad_boxes(Solver):
    from paper_2405_12964_gb300.dwos import DwosError
    sc = scenes.disk_scene("laplace_x", n_query=4)
    s = Solver(0)
    s.load_scene(sc)
    with pytest.raises(DwosError, match="NOT_IMPLEMENTED|mapped"):
        s.boundary_loss_l2([-2, -2], [2, 2])
    sc = scenes.disk_scene("screened_1", n_query=4)
    s.load_scene(sc)
    with pytest.raises(DwosError, match="INVALID_ARG|bad arguments"):
        s.boundary_loss_l2([1, -2], [-1, 2])


def test_general_functional_gradient_is_the_sum_of_its_parts(Solver):
    sc = scenes.disk_scene("screened_1", n_query=4)
    s = Solver(0)
    s.load_scene(sc)
    uref = lambda p: 0.2 * p[:, 0]
    ub = np.full(len(sc.vert), 0.25, np.float32)
    j, g = s.general_functional_gradient([-1, -1], [1, 1], uref, 64, 2000, [-2, -2], [2, 2], ub, seed=3)
    jv, gv = s.functional_gradient([-1, -1], [1, 1], uref, 64, 2000, seed=3)
    jb, gb = s.boundary_loss_l2([-2, -2], [2, 2], ub)
    assert abs(j - (jv + jb)) <= 1e-12 * abs(j)
    assert np.allclose(g, gv + gb, rtol=1e-12, atol=1e-15)
    # g = 1, ub = 1/4 on the 128-gon: J_b = 1/2 (3/4)^2 perimeter, dJ_b/dR = J_b
    n = len(sc.elem)
    assert abs(jb - 0.5 * 0.75 ** 2 * 2 * n * np.sin(np.pi / n)) < 1e-6 * jb
    assert abs(gb[0] - jb) < 1e-6 * jb


def test_boundary_loss_with_host_buffers(Solver):
    # the same call through the C ABI with host target, loss and gradient buffers (mem = host)
    import ctypes
    from paper_2405_12964_gb300 import dwos
    sc = scenes.star_box_scene(n_seg=512, n_query=4)
    s = Solver(0)
    s.load_scene(sc)
    ub = np.linspace(0.0, 1.0, len(sc.vert)).astype(np.float32)
    lo, hi = [-0.7, -1.5], [1.5, 0.4]
    loss_d, g_d = s.boundary_loss_l2(lo, hi, ub)
    lo_c = (ctypes.c_float * 3)(*lo, 0.0)
    hi_c = (ctypes.c_float * 3)(*hi, 0.0)
    loss_h = np.zeros(1, np.float64)
    g_h = np.zeros(s.n_param, np.float64)
    st = dwos.lib().dwos_boundary_loss_l2(s._h, lo_c, hi_c, ub.ctypes.data_as(ctypes.c_void_p),
                                         loss_h.ctypes.data_as(ctypes.c_void_p),
                                         g_h.ctypes.data_as(ctypes.c_void_p), dwos.MEM_HOST)
    assert st == 0, dwos.lib().dwos_last_error(s._h).decode()
    assert abs(loss_h[0] - loss_d) <= 1e-12 * loss_d
    assert np.allclose(g_h, g_d, rtol=1e-12, atol=1e-15)
