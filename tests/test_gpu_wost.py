"""Walks on stars on the GPU (mixed Dirichlet / reflecting Neumann boundaries,
Sec. 3.4 and 4.2) against the FP64 oracle, through the C ABI.

* The K1 of the 2D star weight and the star weight itself against the
  oracle's FP64 definitions (std::cyl_bessel_k and the Green's function flux).
* Per-walk replays of the same Philox walks on the quarter disk (field and
  mapped data), the screened strip, the strip with a source, the slit disk,
  the cube with four Neumann faces and the potential flow past a cylinder: on walks whose branch (steps and
  termination per phase, terminal element) matches, u and udot agree as in the
  Dirichlet parity tests.  Walks end only on Dirichlet elements, numbered as
  the input numbers them.
* Per-point means against the closed forms; the U-statistic gradient and the
  VJP against the oracle's estimators on the same walks.
* The calls that do not support a Neumann part refuse it.
"""
import numpy as np
import pytest
from scipy.special import i0, i1, k0, k1

import oracle
from oracle import closed_forms as cf
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle
from tests.test_gpu_parity import check_walks, run_pair

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


def test_bessel_k1_and_star_weight_match_the_oracle(Solver):
    # K1: A&S 9.8.7 within 8e-9 on x K1 (x <= 2), 9.8.8 within 2.2e-7 on x^(1/2) e^x K1
    # (1.8e-7 relative); FP32 evaluation adds about a dozen roundings
    s = Solver(0)
    # (x <= 80: K1 stays in FP32's normal range)
    x = np.concatenate([np.geomspace(1e-4, 80.0, 3000), [2.0, np.nextafter(2.0, 3.0)]]).astype(np.float32)
    got = s.bessel_k1(x).astype(np.float64)
    want = k1(x.astype(np.float64))
    assert np.all(np.abs(got - want) <= 1.2e-6 * want + 1e-8), (np.abs(got - want) / want).max()
    # star weight: magnitude M of the terms that are summed, argument rounding amplified by 1 + kt + kR;
    # weights below 1e-30 reach FP32's subnormal range and decide Russian roulette against any
    # uniform (>= 2^-24) the same way, hence the absolute floor
    rng = np.random.default_rng(3)
    for dim in (2, 3):
        for sigma in (0.0, 0.3, 4.0, 100.0, 2500.0):
            R = rng.uniform(1e-3, 2.0, 300).astype(np.float32)
            t = (R * rng.uniform(0.001, 1.0, 300)).astype(np.float32)
            w = s.star_weight(dim, sigma, t, R).astype(np.float64)
            k = np.sqrt(float(np.float32(sigma)))
            ref = np.array([oracle.star_weight(dim, float(np.float32(sigma)), float(a), float(b)) for a, b in zip(t, R)])
            kt, kR = k * t.astype(np.float64), k * R.astype(np.float64)
            if dim == 2 and k > 0:
                M = kt * k1(kt) + np.where(kR < 80, kt * i1(kt) * k0(kR) / i0(kR), 0.0)
            else:
                M = ref + 1e-30
            tol = M * (3e-6 + 2.4e-7 * (1 + kt + kR)) + 1e-30
            assert np.all(np.abs(w - ref) <= tol), (dim, sigma, (np.abs(w - ref) / tol).max())


def _replay(Solver, sc, W, differential=True, u_scale=0.0, **opt):
    s, g, o = run_pair(Solver, sc, W, differential=differential, **opt)
    same = check_walks(sc, g, o, differential=differential, max_flip=0.03, u_scale=u_scale)
    dirichlet = np.nonzero(sc.neumann == 0)[0]
    ended = g["rec"]["elem"] >= 0
    assert np.isin(g["rec"]["elem"][ended], dirichlet).all()
    print("%s: %.4f of %d walks on the same branch" % (sc.name, same.mean(), len(same)))
    return s, g, o, same


@pytest.mark.parametrize("data", ["field", "mapped"])
def test_quarter_disk_replay_and_closed_form(Solver, data):
    sc = scenes.quarter_disk_scene(data, n_query=12)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 8192, grad=True)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    ue, due = cf.quarter_disk(sc.query, data)
    assert np.all(np.abs(u - ue) <= 4.5 * use + 3e-3 * np.abs(ue) + 2e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_screened_strip_replay_closed_form_and_reverse_mode(Solver):
    sc = scenes.strip_scene(sigma=4.0, n_query=12, walks=64)
    s, g, o, same = _replay(Solver, sc, 64)
    assert (o["kind"][:, 0] == oracle.KIND_ROULETTE).any()
    out = s.eval(sc.query, 8192, grad=True)
    ue, due = cf.strip(sc.query, 4.0)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 3e-3 * np.abs(ue) + 1e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.01)
    # reverse mode on the same walks: U-statistic gradient, loss and VJP
    n = sc.query.shape[0]
    uref = np.full(n, 0.3)
    loss, gr = (t.cpu().numpy() for t in s.grad_l2(sc.query, uref, sc.walks))
    u_w = np.where(same, o["u_hat"], g["rec"]["u"].astype(np.float64))
    from tests.test_gpu_parity import gpu_udot
    ud_w = np.where(same[:, None], o["udot"], gpu_udot(sc, g["rec"]))
    go = est.grad_l2_ustat(u_w, ud_w, uref, n, sc.walks, 8)
    assert np.allclose(gr, go, rtol=2e-3, atol=2e-3 * np.abs(go).max())
    assert abs(loss[0] - est.loss_l2(u_w, uref, n, sc.walks)) <= 1e-4 * abs(loss[0]) + 1e-7
    w = np.linspace(-1.0, 1.0, n)
    gv = s.vjp(sc.query, w, sc.walks, walk_id_base=0).cpu().numpy()
    vo = est.vjp(ud_w, w, n, sc.walks)
    assert np.allclose(gv, vo, rtol=2e-3, atol=2e-3 * np.abs(vo).max())


def test_strip_with_source_replay_and_closed_form(Solver):
    sc = scenes.strip_scene(sigma=0.0, f=2.0, g=0.5, n_query=12)
    s, g, o, same = _replay(Solver, sc, 64)
    out = s.eval(sc.query, 8192, grad=True)
    ue, due = cf.strip(sc.query, 0.0, f=2.0, g=0.5)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 4e-3 * np.abs(ue) + 2e-3)


def test_slit_disk_replay_and_closed_form(Solver):
    # the slit is a crack: ray parity does not describe this domain, so no inside test
    sc = scenes.slit_disk_scene(n_query=12)
    s, g, o, same = _replay(Solver, sc, 64, differential=False, u_scale=1.0, check_inside=0)
    out = s.eval(sc.query, 8192)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    ue = cf.slit_sqrt(sc.query)
    assert np.all(np.abs(u - ue) <= 4.5 * use + 8e-3)


def test_cube_with_neumann_faces_replay_and_closed_form(Solver):
    sc = scenes.cube_neumann_scene(n_query=8)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 4096, grad=True)
    ue, due = cf.cube_linear(sc.query)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 4e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_cylinder_flow_replay_and_closed_form(Solver):
    # a curved Neumann part: 600 silhouette candidates, searched through their own tree
    sc = scenes.cylinder_flow_scene(n_query=12)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 8192, grad=True)
    ue, due = cf.cylinder_flow(sc.query, sc.meta["a"])
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 2e-3)
    assert np.all(np.abs(du - due) <= 4.5 * dse + 2e-3)


@pytest.mark.parametrize("name", ["slit", "thermal", "cube8"])
def test_walks_on_stars_do_not_depend_on_the_search_order(Solver, name):
    # the Dirichlet tree's search order (per lane: 0; warp-wide: 2; routed: 3, the automatic
    # choice from 128 Dirichlet elements up) changes no walk: records equal bit for bit
    if name == "slit":
        sc, opt, diff = scenes.slit_disk_scene(n_query=8), {"check_inside": 0}, False
    elif name == "thermal":
        sc, opt, diff = scenes.thermal_scene(n_query=8), {}, True
    else:   # 3D, 256 Dirichlet triangles: the automatic order is the warp-wide one
        sc, opt, diff = scenes.cube_neumann_scene(m=8, n_query=8, K=2), {}, True
    recs = []
    for t in (0, 2, 3, -1):
        s = Solver(0)
        s.load_scene(sc, traversal=t, **opt)
        recs.append(s.walk_records(sc.query, 128, walk_id_base=7, differential=diff)["rec"].view(np.uint32))
        s.sync()
    for r in recs[1:]:
        assert np.array_equal(recs[0], r)


@pytest.mark.parametrize("name", ["thermal", "cube"])
def test_walks_on_stars_at_scale_stay_in_the_domain(Solver, name):
    # FP32 walks at scale meet what a few thousand oracle walks do not (rays ending where the
    # sphere touches the Neumann part, tangent moves, convex edges, reflex corners, nested walks
    # starting on a Neumann side, landing points within rounding of the Dirichlet part): over
    # 4 launches of the thermal design (32 x 16384 walks) or the Neumann cube (64 x 4096, K = 2)
    # no walk leaves the domain (a device error) and none reaches the step cap
    if name == "thermal":
        sc = scenes.thermal_scene(n_query=32, walks=16384)
    else:
        sc = scenes.cube_neumann_scene(n_query=64, walks=4096, K=2)
    s = Solver(0)
    s.load_scene(sc)
    total = sc.query.shape[0] * sc.walks
    for i in range(1, 5):
        r = s.walk_records(sc.query, sc.walks, walk_id_base=i * total, differential=True, trace=True)
        s.sync()
        assert s.stats()["capped"] == 0
        tr = r["trace"]
        steps = np.where(tr != 0xFFFFFFFF, tr & 0x3FFFFFFF, 0)
        assert steps.max() < 2000


def test_fine_cube_replay_warp_wide(Solver):
    # the 3D walk-on-stars kernel with the warp-wide search of the Dirichlet tree (256 triangles)
    sc = scenes.cube_neumann_scene(m=8, n_query=8)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 4096, grad=True)
    ue, due = cf.cube_linear(sc.query)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 4e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_sphere_flow_replay_and_closed_form(Solver):
    # a curved Neumann part in 3D (720-triangle icosphere; 768 Dirichlet box triangles: the
    # warp-wide search)
    sc = scenes.sphere_flow_scene(n_query=8)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 8192, grad=True)
    ue, due = cf.sphere_flow(sc.query, sc.meta["a"])
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 3e-3)
    assert np.all(np.abs(du - due) <= 4.5 * dse + 3e-3)


@pytest.mark.parametrize("name", ["sphere", "cylinder"])
def test_normal_cones_change_no_walk(Solver, name):
    # the silhouette query skips tree nodes whose normal cone shows they hold no silhouette (from
    # 1024 candidate elements up, for a fixed Neumann part): the same walks with the cones and
    # without them (a Neumann vertex given a Jacobian column: no cones) are bit-identical
    if name == "sphere":
        sc = scenes.sphere_flow_scene(freq=12, n_query=8)          # 2880 triangles
    else:
        sc = scenes.cylinder_flow_scene(n_circle=2048, n_query=8)
    recs = []
    for moving in (False, True):
        jac = sc.jac
        if moving:
            extra = np.zeros((len(sc.vert), sc.dim, 1))
            extra[sc.elem[np.nonzero(sc.neumann)[0][0], 0], 0, 0] = 1.0
            jac = np.concatenate([sc.jac, extra], axis=2)
        s = Solver(0)
        s.load_scene(sc)
        s.set_boundary(sc.reference_vertices(), sc.elem, jac)
        s.set_neumann(sc.neumann)
        if sc.data == "mapped":
            dg = None if sc.dg_vert is None else np.concatenate([sc.dg_vert, np.zeros((len(sc.vert), 1))], 1) \
                if moving else sc.dg_vert
            s.set_dirichlet_mapped(sc.g_vert, dg)
        recs.append(s.walk_records(sc.query, 256, walk_id_base=11, differential=False)["rec"].view(np.uint32))
        s.sync()
    assert np.array_equal(recs[0], recs[1])


def test_thermal_3d_replay(Solver):
    # the 3D thermal design: query points on the slab's underside (they start on the Neumann
    # part), a Dirichlet sphere and box (368 triangles: the warp-wide search), K = 2
    sc = scenes.thermal_scene_3d(n_side=4)
    sc.query = sc.query.astype(np.float32).astype(np.float64)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    assert np.all(np.isfinite(g["rec"]["u"]))


def test_cones_survive_parameter_updates(Solver):
    # parameter updates refit the trees and rebuild them every 64th time, the candidate tree's
    # normal cones with them: at the same geometry the walks after 65 updates equal the first
    sc = scenes.cylinder_flow_scene(n_circle=2048, n_query=8)
    s = Solver(0)
    s.load_scene(sc)
    first = s.walk_records(sc.query, 128, walk_id_base=3, differential=True)["rec"].view(np.uint32)
    for _ in range(65):
        s.set_params(np.zeros(1))
    again = s.walk_records(sc.query, 128, walk_id_base=3, differential=True)["rec"].view(np.uint32)
    s.sync()
    assert np.array_equal(first, again)


def test_cube_with_a_source_replay_and_closed_form(Solver):
    # the 3D source term of walks on stars (a ball sample counted where x sees it)
    sc = scenes.cube_neumann_scene(n_query=8, f=1.5)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    out = s.eval(sc.query, 4096, grad=True)
    ue, due = cf.cube_linear(sc.query, 1.5)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 5e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_screened_cube_replay_and_closed_form(Solver):
    # the 3D star weight's roulette on the GPU: -u'' + 4 u = 0 on the Neumann cube
    sc = scenes.cube_neumann_scene(n_query=8, sigma=4.0)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    assert (o["kind"][:, 0] == oracle.KIND_ROULETTE).any()
    out = s.eval(sc.query, 4096, grad=True)
    ue, due = cf.cube_screened(sc.query, 4.0)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    assert np.all(np.abs(u - ue) <= 4.5 * use + 4e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_queries_and_refusals_with_a_neumann_part(Solver):
    from paper_2405_12964_gb300.dwos import DwosError
    sc = scenes.quarter_disk_scene("field", n_query=8)
    s = Solver(0)
    s.load_scene(sc)
    rng = np.random.default_rng(4)
    p = rng.uniform(-0.2, 1.2, size=(2000, 2))
    # closest point: the Dirichlet part's, in input numbering
    d, e, _ = (t.cpu().numpy() for t in s.closest_point(p))
    do, _, eo, _ = oracle.closest_point(to_oracle(sc), p)
    assert np.allclose(d, do, rtol=2e-5, atol=2e-6)
    assert np.all(sc.neumann[e] == 0)
    # inside: the whole boundary
    far = oracle.closest_point(oracle.Problem(vert=sc.vert, elem=sc.elem, data_kind="mapped",
                                              g_vert=np.zeros(len(sc.vert))), p)[0] > 1e-4
    gi = s.inside(p).cpu().numpy().astype(bool)
    assert np.array_equal(gi[far], oracle.inside(to_oracle(sc), p)[far])
    with pytest.raises(DwosError):
        s.set_options(dudn_estimator=1)
        s.eval(sc.query, 16, grad=True)
    s.set_options(dudn_estimator=0)
    with pytest.raises(DwosError) as ei:
        s.grad_l2_cv(sc.query, np.zeros(8), 16, cv_grad=np.zeros((8, 2), np.float32))
    assert ei.value.status == 6
    with pytest.raises(DwosError) as ei:
        s.set_neumann(np.ones(len(sc.elem), np.int32))       # no Dirichlet part left
    assert ei.value.status == 1
    s.set_neumann(None)                                     # all Dirichlet again: plain walk on spheres
    s.eval(sc.query, 16)
    s.sync()


@pytest.mark.parametrize("name", ["quarter_disk", "strip", "cube"])
def test_query_points_on_the_neumann_part(Solver, name):
    # points on the Neumann part start their walks on it (normal oriented out of the domain):
    # per-walk replay against the oracle, and the closed forms on that part
    from tests.test_oracle_wost import _on_neumann_points
    sc = _on_neumann_points(name)
    sc.query = sc.query.astype(np.float32).astype(np.float64)     # the same start on both sides
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0)
    assert np.all(np.isfinite(g["rec"]["u"]))
    W = 4096 if name == "cube" else 8192
    out = s.eval(sc.query, W, grad=True)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    if name == "quarter_disk":
        ue, due = cf.quarter_disk(sc.query, "mapped")
    elif name == "strip":
        ue, due = cf.strip(sc.query, 4.0)
    else:
        ue, due = cf.cube_linear(sc.query)
    assert np.all(np.abs(u - ue) <= 4.5 * use + 3e-3 * np.abs(ue) + 4e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.02)


def test_thermal_scene_replay(Solver):
    # the thermal design's scene: a Dirichlet wire under a Neumann slab in a Dirichlet box,
    # differential walks (K = 2) from points on the slab, per walk against the oracle
    sc = scenes.thermal_scene(n_query=8)
    sc.query = sc.query.astype(np.float32).astype(np.float64)
    s, g, o, same = _replay(Solver, sc, 64)
    assert np.all(np.isfinite(g["rec"]["u"]))
    assert (o["kind"][:, 0] == oracle.KIND_SHELL).mean() > 0.99      # sigma = 0: every walk ends in a shell
