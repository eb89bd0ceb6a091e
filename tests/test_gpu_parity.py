"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Per-walk replay: both sides run the same Philox walk ids.  A walk's branch is
(distance queries and termination kind per phase, terminal element).  On
walks whose branch matches, u and the forward-mode derivative agree to 1e-4
relative (absolute floor 1e-5 on u, 1e-3 x (1 + |udot|) on udot, whose
du/dn = (g - u_off)/h carries FP32 rounding of u_off amplified by 1/h); walks
whose branch changed are counted and must be rare.  Means agree within 3.5
combined standard errors.
"""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.golden import philox_kat
from tests.helpers import to_oracle

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


def gpu_udot(sc, rec):
    """Forward-mode udot of each walk rebuilt from its record (see dwos_record)."""
    n = rec.shape[0]
    P = sc.n_param
    out = np.zeros((n, P))
    hit = rec["elem"] >= 0
    e = rec["elem"][hit]
    w = np.stack([1 - rec["b1"][hit] - rec["b2"][hit], rec["b1"][hit], rec["b2"][hit]], 1)
    c = rec["c"][hit].astype(np.float64)[:, :sc.dim]
    acc = np.zeros((hit.sum(), P))
    for i in range(sc.dim):
        v = sc.elem[e, i]
        J = sc.jac[v]                      # (m, dim, P)
        acc += w[:, i:i + 1] * np.einsum("mk,mkp->mp", c, J)
        if sc.dg_vert is not None:
            acc += w[:, i:i + 1] * sc.dg_vert[v]
    out[hit] = acc
    return out


def branch_match(sc, g, o, differential=True):
    K1 = sc.K + 1 if differential else 1
    tr = g["trace"][:, :K1]
    steps_g = (tr & 0x3FFFFFFF).astype(np.int64)
    kind_g = (tr >> 30).astype(np.int64)
    unused = tr == 0xFFFFFFFF
    steps_o = o["steps"][:, :K1].astype(np.int64)
    kind_o = o["kind"][:, :K1].astype(np.int64)
    same = np.ones(tr.shape[0], bool)
    for j in range(K1):
        used_o = kind_o[:, j] >= 0
        same &= (used_o == ~unused[:, j])
        same &= np.where(used_o, (steps_g[:, j] == steps_o[:, j]) & (kind_g[:, j] == kind_o[:, j]), True)
    same &= np.where(kind_o[:, 0] == oracle.KIND_ROULETTE, g["rec"]["elem"] == -1, g["rec"]["elem"] == o["elem"])
    return same


def run_pair(Solver, sc, W, differential=True, base=0, **opt):
    s = Solver(0)
    s.load_scene(sc, **opt)
    g = s.walk_records(sc.query, W, walk_id_base=base, differential=differential, trace=True, debug=True)
    over = {k: v for k, v in opt.items() if k in ("eps", "h", "K", "max_steps", "seed")}
    if "dudn_estimator" in opt:
        over["dudn_mode"] = opt["dudn_estimator"]
    o = oracle.run_walks(to_oracle(sc, **over), sc.query, W, differential=differential, walk_id_base=base)
    return s, g, o


def check_walks(sc, g, o, differential=True, max_flip=0.01, u_scale=0.0):
    """Per-walk agreement on walks whose branch matches.  u_scale: the size of
    the Dirichlet data when it varies continuously along the boundary.  An FP32
    walk ends up to about 1e-4 away from its FP64 replay after tens of steps,
    which moves g(xbar) by |grad g| times that, whatever u's own size (u
    crosses zero where the data does): the 1e-4 bound is then relative to
    |u| + u_scale."""
    same = branch_match(sc, g, o, differential)
    frac_flip = 1 - same.mean()
    assert frac_flip <= max_flip, f"{frac_flip:.4f} of walks changed branch"
    ug = g["rec"]["u"].astype(np.float64)
    uo = o["u_hat"]
    err = np.abs(ug - uo)[same]
    tol = 1e-4 * (np.abs(uo[same]) + u_scale) + 1e-5 + u_drift_allowance(sc, g["rec"], o)[same]
    if sc.f != 0 and sc.neumann is not None:
        # walk on stars with a source: every step's source sample scales with R^2, and R follows
        # the walk's position (the distance to the Dirichlet part or to a silhouette), which in
        # FP32 drifts ~1e-5 from the FP64 replay over tens of steps: the sum of the samples
        # carries that drift; nearly every walk stays within the tight bound, all within 10x
        assert (err <= tol).mean() >= 0.995, (err <= tol).mean()
        assert np.all(err <= 10 * tol), (err / tol).max()
    else:
        assert np.all(err <= tol), (err / tol).max()
    if differential and sc.n_param:
        dg = gpu_udot(sc, g["rec"])
        do = o["udot"]
        e2 = np.abs(dg - do)[same]
        tol = 1e-3 * (1 + np.abs(do[same])) + drift_allowance(sc, g["rec"], o)[same]
        if u_scale > 0 and "debug" in g:
            # continuously varying data: each nested walk drifts like the main walk (its
            # estimate within 1e-4 (|u| + u_scale), as above), and du/dn = (g - u_off) / h
            # carries that into udot times the normal velocity V_n = n . sum_i w_i J_i
            nested = np.abs(normal_velocity(sc, g["rec"], g["debug"])) * (
                1e-4 * (np.abs(g["debug"]["u_off"].astype(np.float64)) + u_scale) / sc.h)[:, None]
            assert (e2 <= tol).mean() >= 0.995, (e2 <= tol).mean()
            tol = tol + nested[same]
        assert np.all(e2 <= tol), (e2 / tol).max()
    return same


def normal_velocity(sc, rec, dbg):
    """V_n = n . sum_i w_i J[v_i] per walk and parameter (0 for walks without a hit)."""
    n, P = rec.shape[0], sc.n_param
    out = np.zeros((n, P))
    hit = rec["elem"] >= 0
    e = rec["elem"][hit]
    w = np.stack([1 - rec["b1"][hit] - rec["b2"][hit], rec["b1"][hit], rec["b2"][hit]], 1).astype(np.float64)
    nrm = dbg["n"][hit].astype(np.float64)[:, :sc.dim]
    acc = np.zeros((hit.sum(), P))
    for i in range(sc.dim):
        acc += w[:, i:i + 1] * np.einsum("mk,mkp->mp", nrm, sc.jac[sc.elem[e, i]])
    out[hit] = acc
    return out


def u_drift_allowance(sc, rec, o):
    """What the measured drift of the end point's vertex weights moves in
    u = sum_i w_i g_i: sum_i |dw_i| |g_i - g_0| over the hit element (field
    data evaluated at its vertices)."""
    n = rec.shape[0]
    out = np.zeros(n)
    hit = (rec["elem"] >= 0) & (o["elem"] >= 0) & (rec["elem"] == o["elem"])
    if not hit.any():
        return out
    e = rec["elem"][hit]
    if sc.data == "field":
        from oracle.closed_forms import harmonic_field
        gv = harmonic_field(sc.vert, sc.field)
    else:
        gv = np.asarray(sc.g_vert, dtype=np.float64)
    g0 = gv[sc.elem[e, 0]]
    acc = np.abs(rec["b1"][hit] - o["bary"][hit, 0]) * np.abs(gv[sc.elem[e, 1]] - g0)
    if sc.dim == 3:
        acc += np.abs(rec["b2"][hit] - o["bary"][hit, 1]) * np.abs(gv[sc.elem[e, 2]] - g0)
    out[hit] = acc
    return out


def drift_allowance(sc, rec, o):
    """What the FP32 end-point drift can move in udot on a matching branch: the
    vertex weights w_i of the hit element differ between the FP32 walk and its
    FP64 replay by the measured |dw_i|, and udot is linear in them with
    coefficients c . J[v_i] + dg[v_i] (see dwos_record).  On short elements a
    1e-4 drift moves w by a few percent, which matters for data derivatives that
    vary from vertex to vertex (random dg); smooth Jacobians hardly see it."""
    n, P = rec.shape[0], sc.n_param
    out = np.zeros((n, P))
    hit = (rec["elem"] >= 0) & (o["elem"] >= 0) & (rec["elem"] == o["elem"])
    e = rec["elem"][hit]
    wg = np.stack([1 - rec["b1"][hit] - rec["b2"][hit], rec["b1"][hit], rec["b2"][hit]], 1).astype(np.float64)
    wo = np.stack([1 - o["bary"][hit, 0] - o["bary"][hit, 1], o["bary"][hit, 0], o["bary"][hit, 1]], 1)
    c = np.abs(rec["c"][hit].astype(np.float64)[:, :sc.dim])
    acc = np.zeros((hit.sum(), P))
    for i in range(sc.dim):
        v = sc.elem[e, i]
        coef = np.einsum("mk,mkp->mp", c, np.abs(sc.jac[v]))
        if sc.dg_vert is not None:
            coef = coef + np.abs(sc.dg_vert[v])
        acc += np.abs(wg[:, i] - wo[:, i])[:, None] * coef
    out[hit] = acc
    return out


def test_philox_bit_exact(Solver):
    s = Solver(0)
    for ctr, key, want in philox_kat():
        got = s.philox(np.array([ctr], dtype=np.uint32), np.array(key, dtype=np.uint32))
        assert [int(x) for x in got[0]] == want
    rng = np.random.default_rng(0)
    ctrs = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x12964, 7], dtype=np.uint32)
    got = s.philox(ctrs, key)
    for i in range(0, 4096, 97):
        assert np.array_equal(got[i], oracle.philox4x32_10(ctrs[i], key))


@pytest.mark.parametrize("traversal", [0, 2, 3])
@pytest.mark.parametrize("which", ["disk", "star", "sphere", "ball_small"])
def test_closest_point_matches_brute_force(Solver, which, traversal):
    rng = np.random.default_rng(1)
    if which == "disk":
        sc = scenes.disk_scene("screened_1")
        p = rng.uniform(-0.95, 0.95, size=(3000, 2))
    elif which == "star":
        sc = scenes.star_box_scene()
        p = rng.uniform(-0.99, 0.99, size=(3000, 2))
    elif which == "sphere":
        sc = scenes.sh_sphere_scene(freq=20, n_query=8)
        p = rng.uniform(-1.9, 1.9, size=(2000, 3))
    else:
        sc = scenes.ball_scene(freq=3)
        p = rng.uniform(-1.2, 1.2, size=(2000, 3))
    s = Solver(0)
    s.load_scene(sc, traversal=traversal)
    d, e, b = (t.cpu().numpy() for t in s.closest_point(p))
    do, xo, eo, bo = oracle.closest_point(to_oracle(sc), p)
    assert np.allclose(d, do, rtol=2e-5, atol=2e-6)
    # The distance is unique; the element is not where two elements are equally
    # close (the closest point is a shared vertex or edge, common outside a finely
    # tessellated convex boundary).  Where the ids differ, the GPU's element must be
    # exactly as close and the oracle's closest point must lie on its element's border.
    dis = np.nonzero(e != eo)[0]
    pr = to_oracle(sc)
    for i in dis:
        one = oracle.Problem(vert=sc.vert, elem=sc.elem[e[i]:e[i] + 1], data_kind="mapped",
                             g_vert=np.zeros(len(sc.vert)))
        dg = oracle.closest_point(one, p[i:i + 1])[0][0]
        # exactly as close up to FP32 rounding of coordinates and distances
        assert abs(dg - do[i]) <= 4e-7 * max(1.0, float(np.abs(p[i]).max())) + 2e-7 * do[i] + 1e-7, (dg, do[i])
    assert len(dis) <= 0.5 * len(p)


def test_inside_test_matches_oracle(Solver):
    rng = np.random.default_rng(2)
    sc = scenes.star_box_scene(n_seg=1024)
    p = rng.uniform(-1.2, 1.2, size=(4000, 2))
    s = Solver(0)
    s.load_scene(sc)
    gi = s.inside(p).cpu().numpy().astype(bool)
    oi = oracle.inside(to_oracle(sc), p)
    dist = oracle.closest_point(to_oracle(sc), p)[0]
    far = dist > 1e-4
    assert np.array_equal(gi[far], oi[far])
    sc3 = scenes.sh_sphere_scene(freq=12, n_query=8)
    p3 = rng.uniform(-2.2, 2.2, size=(1500, 3))
    s.load_scene(sc3)
    gi = s.inside(p3).cpu().numpy().astype(bool)
    oi = oracle.inside(to_oracle(sc3), p3)
    far = oracle.closest_point(to_oracle(sc3), p3)[0] > 1e-4
    assert np.array_equal(gi[far], oi[far])


@pytest.mark.parametrize("variant", ["screened_1", "laplace_x", "mapped_cos"])
def test_disk_per_walk_replay(Solver, variant):
    sc = scenes.disk_scene(variant, n_query=16)
    s, g, o = run_pair(Solver, sc, 96)
    check_walks(sc, g, o)


@pytest.mark.parametrize("traversal", [0, 2, 3])
def test_star_box_per_walk_replay_with_nested_walks(Solver, traversal):
    sc = scenes.star_box_scene(n_seg=4096, n_query=24)
    s, g, o = run_pair(Solver, sc, 32, K=2, traversal=traversal)
    same = check_walks(sc, g, o)
    # debug outputs: du/dn and the oracle's agree on matching walks
    dd = g["debug"]["dudn"].astype(np.float64)
    assert np.all(np.abs(dd - o["dudn"])[same] <= 1e-3 * (1 + np.abs(o["dudn"][same])))


@pytest.mark.parametrize("which", ["star", "sphere"])
def test_ball_gradient_estimator_replay(Solver, which):
    # Eq. (dudn_mc_estimate): each nested walk's first move samples the sphere about
    # the offset point (no roulette, no source) and weighs the estimate at y
    if which == "star":
        sc = scenes.star_box_scene(n_seg=4096, n_query=16)
        s, g, o = run_pair(Solver, sc, 32, K=2, dudn_estimator=1)
    else:
        sc = scenes.sh_sphere_scene(freq=16, n_query=12, K=2)
        s, g, o = run_pair(Solver, sc, 24, dudn_estimator=1)
    same = check_walks(sc, g, o, max_flip=0.02)
    dd = g["debug"]["dudn"].astype(np.float64)
    assert np.all(np.abs(dd - o["dudn"])[same] <= 1e-3 * (1 + np.abs(o["dudn"][same])))
    assert np.abs(o["dudn"][same]).max() > 0


@pytest.mark.parametrize("traversal", [0, 2, 3])
def test_sphere_3d_per_walk_replay_with_source(Solver, traversal):
    sc = scenes.sh_sphere_scene(freq=16, n_query=12, K=2)
    s, g, o = run_pair(Solver, sc, 24, traversal=traversal)
    check_walks(sc, g, o, max_flip=0.02)


def test_warp_wide_search_is_the_one_that_ran(Solver):
    # same walks, same results; the 32-wide tree needs far fewer node visits
    sc = scenes.sh_sphere_scene(freq=40, n_query=64)
    out, nodes = [], []
    for t in (0, 2):
        s = Solver(0)
        s.load_scene(sc, traversal=t)
        out.append(s.walk_records(sc.query, 64)["rec"])
        st = s.stats()
        nodes.append((st["nodes_visited"] + st["wide_nodes_visited"]) / (st["steps_main"] + st["steps_nested"]))
    info = s.bvh_info()
    fill = (info["n_wide"] - 1 + info["n_tree"]) / (32.0 * info["n_wide"])
    print("32-wide tree: %d nodes, %d levels, %.2f of the child slots used" % (info["n_wide"], info["wide_depth"], fill))
    assert info["n_tree"] + info["n_big"] == info["n_elem"] and fill > 0.5
    same = out[0]["elem"] == out[1]["elem"]
    assert same.mean() > 0.99
    assert np.allclose(out[0]["u"][same], out[1]["u"][same], rtol=1e-5, atol=1e-6)
    print("node visits per query: binary %.1f, 32-wide %.1f" % tuple(nodes))
    assert nodes[1] < 0.5 * nodes[0]


def test_routed_search_skips_the_tree_and_keeps_the_walks(Solver):
    # order 3: every query tests the binary root's two child boxes against its bound (one
    # node visit); only the queries that reach inside them are searched, over the 32-wide
    # tree; the closest element, hence every walk, is the same as with order 0
    sc = scenes.star_box_scene(n_query=32, walks=256)
    out, st = [], []
    for t in (0, 3):
        s = Solver(0)
        s.load_scene(sc, traversal=t)
        out.append(s.walk_records(sc.query, sc.walks)["rec"])
        st.append(s.stats())
    steps = [x["steps_main"] + x["steps_nested"] for x in st]
    assert st[0]["wide_nodes_visited"] == 0 and st[1]["wide_nodes_visited"] > 0
    assert st[1]["nodes_visited"] >= steps[1]
    # most queries stop at the root test: far fewer node visits than the per-lane search
    assert st[1]["wide_nodes_visited"] < 0.25 * steps[1]
    same = out[0]["elem"] == out[1]["elem"]
    assert same.mean() > 0.99
    assert np.allclose(out[0]["u"][same], out[1]["u"][same], rtol=1e-5, atol=1e-6)


def test_replay_from_points_at_and_near_the_shell(Solver):
    # query points at 0.5, 2 and 5 eps from the boundary (inside): the first query may end the
    # walk at once; u and udot must still match the oracle walk for walk
    sc = scenes.disk_scene("screened_1", n_query=4)
    n = len(sc.elem)
    apothem = np.cos(np.pi / n)
    t = (np.arange(48) + 0.37) * (2 * np.pi / 48)        # off the polygon's vertex rays (exact ties)
    q = []
    for dd in (0.5, 2.0, 5.0):
        r = apothem - dd * sc.eps
        q.append(np.stack([r * np.cos(t), r * np.sin(t)], 1))
    sc.query = np.concatenate(q)
    s, g, o = run_pair(Solver, sc, 32)
    same = check_walks(sc, g, o, max_flip=0.02)
    print("near-shell replay: %.4f of walks on the same branch" % same.mean())


def test_forward_only_walks_match(Solver):
    sc = scenes.ball_scene(freq=8, n_query=10, sigma=2.0, f=0.7)
    s, g, o = run_pair(Solver, sc, 64, differential=False)
    check_walks(sc, g, o, differential=False)


def test_walk_id_base_replays_subsets(Solver):
    sc = scenes.disk_scene("screened_1", n_query=6)
    s = Solver(0)
    s.load_scene(sc)
    a = s.walk_records(sc.query, 64)["rec"]
    b = s.walk_records(sc.query[3:4], 64, walk_id_base=3 * 64)["rec"]
    assert np.array_equal(a[192:256].view(np.uint8), b.view(np.uint8))


def test_eval_means_match_oracle_and_closed_form(Solver):
    sc = scenes.disk_scene("screened_1", n_query=64, walks=1024)
    s = Solver(0)
    s.load_scene(sc)
    out = s.eval(sc.query, sc.walks, grad=True)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    o = oracle.run_walks(to_oracle(sc), sc.query, sc.walks, differential=True)
    uo, uose = est.point_mean_se(o["u_hat"], 64, sc.walks)
    duo, duose = est.point_mean_se(o["udot"], 64, sc.walks)
    # same walks: the per-point means are nearly identical, far inside 3.5 SE
    assert np.all(np.abs(u - uo) <= 3.5 * np.sqrt(use ** 2 + uose ** 2) / 4 + 1e-6)
    assert np.all(np.abs(du - duo) <= 3.5 * np.sqrt(dse ** 2 + duose ** 2) / 4 + 1e-6)
    assert np.allclose(use, uose, rtol=0.05, atol=1e-6)
    # 64 points x 18 quantities: 4.5 SE keeps the family-wise false-alarm rate small.
    # With g = 1 a nested walk returns exactly g unless roulette stops it, so du/dn is a
    # rare-event estimate (a handful of nonzero walks per point) whose per-point sample SE
    # is unreliable; the median SE over the points stands in where it is larger.
    ue, due = cf.disk_screened_const(sc.query, 1.0, 4.0)
    assert np.all(np.abs(u - ue) <= 4.5 * use + 2e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.01)


def test_grad_l2_and_vjp_match_oracle_estimators(Solver):
    sc = scenes.star_box_scene(n_seg=1024, n_query=16, walks=64)
    s = Solver(0)
    s.load_scene(sc, K=2)
    uref = sc.u_ref
    loss, g = (t.cpu().numpy() for t in s.grad_l2(sc.query, uref, sc.walks))
    o = oracle.run_walks(to_oracle(sc, K=2), sc.query, sc.walks, differential=True)
    go = est.grad_l2_ustat(o["u_hat"], o["udot"], uref, 16, sc.walks, 8)
    lo = est.loss_l2(o["u_hat"], uref, 16, sc.walks)
    scale = np.abs(go).max()
    assert np.allclose(g, go, rtol=2e-3, atol=2e-3 * scale), np.abs(g - go).max() / scale
    assert abs(loss[0] - lo) <= 1e-4 * abs(lo) + 1e-7
    w = np.linspace(-1, 1, 16)
    gv = s.vjp(sc.query, w, sc.walks, walk_id_base=0).cpu().numpy()
    vo = est.vjp(o["udot"], w, 16, sc.walks)
    assert np.allclose(gv, vo, rtol=2e-3, atol=2e-3 * np.abs(vo).max())


def test_product_estimators_match_oracle(Solver):
    # Sec. 4.3: U-statistic (= dwos_grad_l2), correlated and uncorrelated products on the same walks
    sc = scenes.star_box_scene(n_seg=1024, n_query=16, walks=64)
    s = Solver(0)
    s.load_scene(sc, K=2)
    uref = sc.u_ref
    o = oracle.run_walks(to_oracle(sc, K=2), sc.query, sc.walks, differential=True)
    want = {"ustat": est.grad_l2_ustat(o["u_hat"], o["udot"], uref, 16, sc.walks, 8),
            "correlated": est.grad_l2_correlated(o["u_hat"], o["udot"], uref, 16, sc.walks),
            "uncorrelated": est.grad_l2_uncorrelated(o["u_hat"], o["udot"], uref, 16, sc.walks)}
    lo = est.loss_l2(o["u_hat"], uref, 16, sc.walks)
    for name, go in want.items():
        loss, g = (t.cpu().numpy() for t in s.grad_l2_product(sc.query, uref, sc.walks, product=name))
        scale = np.abs(go).max()
        assert np.allclose(g, go, rtol=2e-3, atol=2e-3 * scale), (name, np.abs(g - go).max() / scale)
        assert abs(loss[0] - lo) <= 1e-4 * abs(lo) + 1e-7
    g1 = s.grad_l2(sc.query, uref, sc.walks)[1].cpu().numpy()
    g2 = s.grad_l2_product(sc.query, uref, sc.walks, product="ustat")[1].cpu().numpy()
    assert np.allclose(g1, g2, rtol=1e-9, atol=1e-12 * np.abs(g1).max())     # FP64 atomics: order may differ


def test_vertex_gradient_chains_to_parameters(Solver):
    sc = scenes.star_box_scene(n_seg=512, n_query=8, walks=64)
    s = Solver(0)
    s.load_scene(sc)
    loss, g, gv = s.grad_l2(sc.query, sc.u_ref, sc.walks, vertex_grad=True)
    g, gv = g.cpu().numpy(), gv.cpu().numpy()
    chained = np.einsum("vk,vkp->p", gv, sc.jac)
    # the library holds J in FP32; the chain rule here uses the FP64 scene Jacobian
    assert np.allclose(g, chained, rtol=2e-5, atol=1e-6 * np.abs(g).max())


# ---------------------------------------------------------------- edge cases
def test_edge_cases(Solver):
    import torch
    from paper_2405_12964_gb300.dwos import DwosError
    sc = scenes.disk_scene("screened_1", n_query=4)
    s = Solver(0)
    s.load_scene(sc)
    out = s.eval(np.zeros((0, 2)), 16)
    assert out["u"].numel() == 0
    out = s.eval(sc.query, 1)
    assert np.all(out["u_se"].cpu().numpy() == 0)
    # a point inside the shell stops at once: u = g(xbar) exactly
    r = s.walk_records(np.array([[0.9995, 0.0]]), 4, trace=True)
    assert np.all(r["rec"]["u"] == 1.0) and np.all((r["trace"][:, 0] & 0x3FFFFFFF) == 1)
    # outside the domain: loud error
    with pytest.raises(DwosError) as ei:
        s.eval(np.array([[1.5, 0.0]]), 8)
        torch.cuda.synchronize()
        s.sync()
    assert ei.value.status == 8
    # invalid options
    with pytest.raises(DwosError):
        s.set_options(B=3)
    with pytest.raises(DwosError):
        s.set_options(eps=0.0)
    s.set_options(eps=1e-3, B=8)
    # grad_l2 needs W % B == 0
    with pytest.raises(DwosError):
        s.grad_l2(sc.query, np.zeros(4), 12)


def test_offset_inside_shell_gives_zero_derivative_on_gpu(Solver):
    sc = scenes.disk_scene("screened_1", n_query=6)
    s = Solver(0)
    s.load_scene(sc, h=5e-4)
    out = s.eval(sc.query, 256, grad=True)
    assert np.all(out["du"].cpu().numpy() == 0.0)


def test_single_element_and_tiny_meshes(Solver):
    # one triangle far away plus checks of the single-leaf BVH
    vert = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    s = Solver(0)
    s.set_boundary(vert, np.array([[0, 1, 2]], dtype=np.int32))
    p = np.array([[0.2, 0.2, 0.5], [2.0, 2.0, 2.0], [-1.0, 0.3, 0.0]])
    d, e, b = (t.cpu().numpy() for t in s.closest_point(p))
    pr = oracle.Problem(vert=vert, elem=np.array([[0, 1, 2]], np.int32), data_kind="mapped", g_vert=np.zeros(3))
    do = oracle.closest_point(pr, p)[0]
    assert np.allclose(d, do, rtol=1e-6) and np.all(e == 0)


def test_capped_walks_are_counted(Solver):
    sc = scenes.disk_scene("screened_1", n_query=4)
    s = Solver(0)
    s.load_scene(sc, max_steps=3)
    s.set_pde(0.0, 0.0)
    g = s.walk_records(sc.query, 64, trace=True)
    st = s.stats()
    assert st["capped"] > 0
    o = oracle.run_walks(to_oracle(sc, max_steps=3, sigma=0.0), sc.query, 64, differential=True)
    capped_o = (o["kind"] == oracle.KIND_CAPPED).sum()
    assert abs(int(st["capped"]) - int(capped_o)) <= 2
    assert ((g["trace"][:, 0] & 0x3FFFFFFF) <= 3).all()


@pytest.mark.parametrize("traversal", [0, 1, 2, 3])
@pytest.mark.parametrize("which", ["star", "sphere"])
def test_hinted_closest_point_equals_unhinted(Solver, which, traversal):
    # the walk seeds each query with the previous hit and climbs the BVH from it,
    # stopping at the first Morton cell that contains the search ball; with any
    # hint (good, random, or none) the distance must be the brute-force minimum
    rng = np.random.default_rng(5)
    if which == "star":
        sc = scenes.star_box_scene()
        p = rng.uniform(-0.99, 0.99, size=(4000, 2))
    else:
        sc = scenes.sh_sphere_scene(freq=40, n_query=8)
        p = rng.uniform(-1.95, 1.95, size=(3000, 3))
    s = Solver(0)
    s.load_scene(sc, traversal=traversal)
    d0, e0, _ = (t.cpu().numpy() for t in s.closest_point(p))
    hints = {
        "random": rng.integers(0, sc.elem.shape[0], size=len(p)),
        "own": e0,
        "none": np.full(len(p), -1),
    }
    # a nearby element: the closest element of a slightly moved point
    d1, e1, _ = (t.cpu().numpy() for t in s.closest_point(p + 0.05 * rng.normal(size=p.shape)))
    hints["near"] = e1
    for name, h in hints.items():
        d, e, b = (t.cpu().numpy() for t in s.closest_point_hint(p, h.astype(np.int32)))
        assert np.allclose(d, d0, rtol=1e-6, atol=1e-7), (name, np.abs(d - d0).max())
    do = oracle.closest_point(to_oracle(sc), p[:500])[0]
    assert np.allclose(d0[:500], do, rtol=2e-5, atol=2e-6)


def test_inside_test_is_watertight_on_fine_boundaries(Solver):
    # very short segments / small triangles: a ray through a shared vertex or
    # edge must count one crossing, never zero or two
    s = Solver(0)
    st = scenes.star_box_scene(n_seg=400_000, n_query=2048)
    s.load_scene(st)
    assert np.all(s.inside(st.query).cpu().numpy() == 1)
    rng = np.random.default_rng(9)
    a = rng.uniform(0, 2 * np.pi, 4000)
    inner = np.stack([0.1 * np.cos(a), 0.1 * np.sin(a)], 1)          # inside the star: outside Omega
    assert np.all(s.inside(inner).cpu().numpy() == 0)
    sp = scenes.sh_sphere_scene(freq=120, n_query=2048)
    s.load_scene(sp)
    assert np.all(s.inside(sp.query).cpu().numpy() == 1)
    d = rng.normal(size=(4000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    assert np.all(s.inside(0.5 * d).cpu().numpy() == 0)


def test_walks_do_not_depend_on_search_order_or_schedule(Solver):
    # walks that end at a vertex shared by two segments tie exactly; the search breaks the tie
    # the same way in every order (lower leaf index, boxes searched up to a 1e-5 margin over
    # the bound), so the records are bit-identical across orders and repeated runs
    sc = scenes.star_box_scene(n_seg=1024, n_query=4)
    s = Solver(0)
    s.load_scene(sc, K=2)
    pts, _ = s.sample_domain(200, [-0.8, -0.8], [0.8, 0.8], seed=5)
    recs = []
    for t in (0, 2, 3, 3):
        s = Solver(0)
        s.load_scene(sc, K=2, traversal=t)
        recs.append(s.walk_records(pts, 64)["rec"].view(np.uint32))
    for r in recs[1:]:
        assert np.array_equal(recs[0], r)


def test_routed_search_per_lane_branch_on_a_disk(Solver):
    # on the 128-gon every element is in the tree, so every query reaches inside the root's
    # boxes and full warps take order 3's per-lane branch (more than 16 lanes need a search);
    # the walks must equal those of the per-lane (0) and warp-wide (2) orders bit for bit
    sc = scenes.disk_scene("screened_1", n_query=64)
    recs, st = [], []
    for t in (0, 2, 3):
        s = Solver(0)
        s.load_scene(sc, traversal=t)
        recs.append(s.walk_records(sc.query, 512)["rec"].view(np.uint32))
        st.append(s.stats())
    steps = st[2]["steps_main"] + st[2]["steps_nested"]
    # one root test per query, plus the per-lane branch's binary fetches
    assert st[2]["nodes_visited"] > 2 * steps
    assert np.array_equal(recs[0], recs[1]) and np.array_equal(recs[0], recs[2])
