"""Learned control variate on the 2D shape-from-diffusion geometry.

The walk estimate of u at a query point x0 is corrected by the network's
gradient: u - grad u~(x0) . (x1 - x0), where x1 is the main walk's first step
(the direction is uniform and independent of the roulette draw), so the
correction has mean zero for any network.  Checks: the per-walk corrected
estimates and the U-statistic loss gradient equal the oracle's on the same
walks and the same cv gradient; the correction is zero-mean; a network trained
on the walks' own samples reduces the variance of u.
"""
import numpy as np
import pytest

import oracle
from oracle.cv import nested_cv_table
from oracle import estimators as est
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    return torch, dwos


def _corrected(o, xq, W, g, whole=False):
    x1 = (o["x_end"] if whole else o["x1"])[:, :2]
    moved = ~np.isnan(x1[:, 0])
    p = np.repeat(np.arange(xq.shape[0]), W)
    corr = np.zeros(len(p))
    corr[moved] = ((x1[moved] - xq[p[moved]]) * g[p[moved]]).sum(1)
    return o["u_hat"] - corr


@pytest.mark.parametrize("whole", [False, True])
def test_cv_gradient_matches_oracle_on_the_same_walks(env, whole):
    torch, dwos = env
    sc = scenes.star_box_scene(n_seg=1024, n_query=12, walks=64)
    s = dwos.Solver(0)
    s.load_scene(sc)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(12, 2)).astype(np.float32)
    out = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, walk_id_base=0, cv_grad=g, whole_walk=whole, samples=True)
    o = oracle.run_walks(to_oracle(sc), sc.query, sc.walks, differential=True)
    uc = _corrected(o, sc.query, sc.walks, g.astype(np.float64), whole)
    go = est.grad_l2_ustat(uc, o["udot"], sc.u_ref, 12, sc.walks, 8)
    gg = out["grad"].cpu().numpy()
    assert np.allclose(gg, go, rtol=2e-3, atol=2e-3 * np.abs(go).max())
    lo = est.loss_l2(uc, sc.u_ref, 12, sc.walks)
    assert abs(float(out["loss"][0]) - lo) <= 1e-4 * abs(lo) + 1e-7
    # samples: x1 and the estimate of u at x1 (u minus the first ball's source, zero here)
    smp = out["samples"].cpu().numpy()
    moved = ~np.isnan(o["x1"][:, 0])
    assert np.array_equal(~np.isnan(smp[:, 0]), moved)
    assert np.allclose(smp[moved, :2], o["x1"][moved, :2], atol=1e-5)
    assert np.allclose(smp[moved, 3], o["u_hat"][moved], atol=1e-5)


def test_correction_has_zero_mean(env):
    torch, dwos = env
    sc = scenes.star_box_scene(n_query=64, walks=4096)
    s = dwos.Solver(0)
    s.load_scene(sc)
    rng = np.random.default_rng(4)
    g = rng.normal(size=(64, 2)).astype(np.float32) * 3.0
    out = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, cv_grad=g, samples=True)
    smp = out["samples"].cpu().numpy()
    W = sc.walks
    moved = ~np.isnan(smp[:, 0])
    p = np.repeat(np.arange(64), W)
    corr = np.zeros(len(p))
    corr[moved] = ((smp[moved, :2] - sc.query[p[moved]]) * g[p[moved]]).sum(1)
    c = corr.reshape(64, W)
    z = c.mean(1) / (c.std(1, ddof=1) / np.sqrt(W))
    assert np.abs(z).max() < 4.5
    assert abs(z.mean()) < 4.0 / np.sqrt(64)


def test_exact_gradient_removes_the_variance_of_linear_data(env):
    # sigma = 0, g = x: u = x is linear, so u - (1, 0) . (x_end - x0) equals
    # x0 up to the eps-shell offset: the whole-walk correction leaves almost no
    # variance, the first-step one removes the first step's share
    torch, dwos = env
    sc = scenes.disk_scene("laplace_x", n_query=32, walks=2048)
    s = dwos.Solver(0)
    s.load_scene(sc)
    g = np.tile([[1.0, 0.0]], (32, 1)).astype(np.float32)
    uref = np.zeros(32)
    whole = s.grad_l2_cv(sc.query, uref, sc.walks, cv_grad=g, whole_walk=True)
    first = s.grad_l2_cv(sc.query, uref, sc.walks, cv_grad=g)
    r_whole = (whole["u_se_cv"] / whole["u_se"]).cpu().numpy() ** 2
    r_first = (first["u_se_cv"] / first["u_se"]).cpu().numpy() ** 2
    assert np.all(r_whole < 0.01), r_whole.max()
    assert np.all(r_first < 1.0) and np.median(r_first) < 0.8, np.median(r_first)


def test_trained_network_reduces_variance(env):
    torch, dwos = env
    sc = scenes.star_box_scene(n_query=256, walks=1024)
    s = dwos.Solver(0)
    s.load_scene(sc)
    net = dwos.ControlVariateNet(seed=1)
    # fit u on the walks' own first-step samples (x1, estimate of u at x1)
    for it in range(6):
        out = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, walk_id_base=(it + 1) << 24, samples=True)
        smp = out["samples"]
        ok = ~torch.isnan(smp[:, 0])
        x = smp[ok, :2].contiguous()
        t = torch.stack([smp[ok, 3], torch.zeros_like(smp[ok, 3])], 1).contiguous()
        m = torch.stack([torch.ones_like(t[:, 0]), torch.zeros_like(t[:, 0])], 1).contiguous()
        for _ in range(60):
            net.train_step(x, t, m, lr=2e-3)
    _, grad_u, _ = net.eval(sc.query)
    plain = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, walk_id_base=99 << 24)
    first = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, walk_id_base=99 << 24, cv_grad=grad_u)
    whole = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, walk_id_base=99 << 24, cv_grad=grad_u, whole_walk=True)
    r_first = (first["u_se_cv"] / plain["u_se"]).cpu().numpy() ** 2
    r_whole = (whole["u_se_cv"] / plain["u_se"]).cpu().numpy() ** 2
    print("variance ratio with the learned control variate: first step %.3f, whole walk %.3f"
          % (np.median(r_first), np.median(r_whole)))
    assert np.median(r_first) < 1.0
    assert np.median(r_whole) < 0.85, np.median(r_whole)
    # same walks: the plain SE column of the CV call equals the plain call's
    assert np.allclose(first["u_se"].cpu().numpy(), plain["u_se"].cpu().numpy())


def test_nested_cv_table_matches_oracle(env):
    # the per-element table (q, t) corrects each nested walk by (q n + t) . (x_end - x_off)
    torch, dwos = env
    from tests.test_gpu_parity import branch_match
    sc = scenes.star_box_scene(n_seg=1024, n_query=12, walks=64)
    s = dwos.Solver(0)
    s.load_scene(sc)
    rng = np.random.default_rng(5)
    tab = rng.normal(size=(sc.elem.shape[0], 4)).astype(np.float32)
    g = rng.normal(size=(12, 2)).astype(np.float32)
    recs = s.walk_records(sc.query, sc.walks, trace=True)         # the table changes no walk's path
    out = s.grad_l2_cv(sc.query, sc.u_ref, sc.walks, cv_grad=g, whole_walk=True, cv_elem=tab, debug=True)
    o = oracle.run_walks(to_oracle(sc, cv_elem=tab.astype(np.float64)), sc.query, sc.walks, differential=True)
    same = branch_match(sc, recs, o)
    assert same.mean() > 0.97
    dbg = out["debug"].view(torch.float32).view(-1, 12).cpu().numpy().astype(np.float64)
    dd = dbg[:, 0]
    # The correction is continuous in the walk positions, so unlike u (piecewise-constant
    # data) it also shows how far the FP32 walk drifted from the FP64 one.  The ball-step map
    # amplifies rounding (near corners by up to ~2x per step), so a walk with the same branch
    # can end 1e-4 away.  Tight check on walks whose main walk ends where the oracle's does;
    # the nested walks' own drift (a few 1e-7 per step) scales with |q n + t| / (K h).
    tight = same & (np.abs(dbg[:, 5:7] - o["xbar"][:, :2]).max(1) < 1e-5)
    assert tight.mean() > 0.9, tight.mean()
    K = sc.K
    nested_steps = (recs["trace"][:, 1:K + 1] & 0x3FFFFFFF).astype(np.float64)
    nested_steps[recs["trace"][:, 1:K + 1] == 0xFFFFFFFF] = 0
    gmax = np.abs(tab.astype(np.float64)).sum(1)[np.maximum(o["elem"], 0)]
    drift = gmax * (1e-6 + 5e-7 * nested_steps.sum(1)) / (K * sc.h)
    err = np.abs(dd - o["dudn"])
    tol = 1e-3 * (1 + np.abs(o["dudn"])) + drift
    ok = err <= tol
    print("nested cv parity: %d tight walks of %d, %.4f within tolerance, median err %.3g, max err/tol %.3g"
          % (tight.sum(), tight.size, ok[tight].mean(), np.median(err[tight]), (err / tol)[tight].max()))
    assert ok[tight].mean() >= 0.98
    assert np.median(err[tight]) < 1e-4
    # the record's parts: uncorrected nested mean and the mean displacements
    pos = 2e-6 + 5e-7 * nested_steps.sum(1)
    for name, col, scale in (("u_plain", 8, 1e-5), ("disp_n", 9, 0.0), ("disp_t", 10, 0.0)):
        lim = scale + pos * (gmax if name == "disp_t" else 1.0)
        okp = np.abs(dbg[:, col] - o[name]) <= lim
        assert okp[tight].mean() >= 0.98, name
    elem_gpu = out["debug"].view(torch.int32).view(-1, 12)[:, 11].cpu().numpy()
    assert np.array_equal(elem_gpu[same], o["elem"][same])
    uc = _corrected(o, sc.query, sc.walks, g.astype(np.float64), True)
    go = est.grad_l2_ustat(uc, o["udot"], sc.u_ref, 12, sc.walks, 8)
    gg = out["grad"].cpu().numpy()
    assert np.allclose(gg, go, rtol=2e-3, atol=2e-3 * np.abs(go).max())


def test_exact_boundary_gradient_collapses_nested_variance(env):
    # u = x: q = n_x and t = e_x - n_x n give grad u exactly; du/dn keeps only the eps-shell offset
    torch, dwos = env
    sc = scenes.disk_scene("laplace_x", n_query=32, walks=1024)
    s = dwos.Solver(0)
    s.load_scene(sc)
    v, e = sc.vert, sc.elem
    d = v[e[:, 1]] - v[e[:, 0]]
    n = np.stack([d[:, 1], -d[:, 0]], 1) / np.linalg.norm(d, axis=1)[:, None]
    n *= np.sign(((v[e[:, 0]] + v[e[:, 1]]) * n).sum(1))[:, None]
    tab = nested_cv_table(v, e, v[:, 0], n[:, 0])
    uref = np.zeros(32)
    res = []
    for t in (None, tab):
        out = s.grad_l2_cv(sc.query, uref, sc.walks, cv_elem=t, debug=True)
        rec = out["debug"].view(torch.float32).view(-1, 12).cpu().numpy().astype(np.float64)
        hit = (rec[:, 1] != 0) | (rec[:, 2] != 0)
        res.append(rec[hit, 0] - rec[hit, 1])                      # du/dn minus the closed form n_x
    ratio = res[1].var() / res[0].var()
    print("nested du/dn variance ratio with the exact table: %.2e" % ratio)
    assert ratio < 0.01, ratio
    assert abs(res[1].mean()) < 0.05


def test_cv_table_matches_host_reference(env):
    # dwos_cv_table: the du/dn head at element centres and the data's tangential gradient
    torch, dwos = env
    net = dwos.ControlVariateNet(seed=3)
    s = dwos.Solver(0)
    for sc, g in ((scenes.star_box_scene(n_seg=1024, n_query=8), None),
                  (scenes.disk_scene("laplace_x", n_query=8), "x")):
        s.load_scene(sc)
        tab = s.cv_table(net).cpu().numpy()
        centres = (0.5 * (sc.vert[sc.elem[:, 0]] + sc.vert[sc.elem[:, 1]])).astype(np.float32)
        q = net.eval(centres)[2].cpu().numpy()
        g_vert = sc.vert[:, 0] if g == "x" else sc.g_vert       # g = x is linear: its tangential gradient is exact
        ref = nested_cv_table(sc.vert, sc.elem, g_vert, q)
        assert np.allclose(tab, ref, rtol=1e-4, atol=1e-5), np.abs(tab - ref).max()


def test_cv_training_set_matches_its_definition(env):
    # dwos_cv_training_set: the network's training rows built on the device from one
    # dwos_grad_l2_cv call's per-walk samples and debug records, against the rows
    # written out here from the same per-walk values
    torch, dwos = env
    sc = scenes.star_box_scene(n_seg=1024, n_query=16, walks=64)
    s = dwos.Solver(0)
    s.load_scene(sc)
    net = dwos.ControlVariateNet(seed=2)
    xq = torch.tensor(sc.query, dtype=torch.float32, device="cuda")
    out = s.grad_l2_cv(xq, sc.u_ref, sc.walks, cv_grad=net.eval(xq)[1], whole_walk=True, cv_elem=s.cv_table(net),
                       samples=True, debug=True)
    smp = out["samples"].cpu().numpy().astype(np.float64)
    dbg = out["debug"].view(torch.float32).view(-1, 12).cpu().numpy().astype(np.float64)
    n = smp.shape[0]
    for stride, off, qw in ((1, 0, 0.2), (3, 2, 0.5)):
        x, t, m = (a.cpu().numpy().astype(np.float64) for a in s.cv_training_set(out["samples"], out["debug"],
                                                                                 stride, off, qw))
        idx = np.arange(off, n, stride)
        R = len(idx)
        assert x.shape == (2 * R, 2)
        sm, d = smp[idx], dbg[idx]
        ok = ~np.isnan(sm[:, 0])
        assert np.array_equal(x[:R][ok], sm[ok, :2]) and np.all(x[:R][~ok] == 0)
        assert np.array_equal(t[:R, 0][ok], sm[ok, 3]) and np.all(t[:R, 1] == 0)
        assert np.array_equal(m[:R, 0], ok.astype(float)) and np.all(m[:R, 1] == 0)
        dudn, nx, ny, u_off, xb, u_plain, dn, dt = d[:, 0], d[:, 1], d[:, 2], d[:, 4], d[:, 5:7], d[:, 8], d[:, 9], d[:, 10]
        hit = ((nx != 0) | (ny != 0)) & (np.abs(dn) > 1e-7)
        res = np.where(hit, u_plain - (u_off + sc.h * dudn) - dt, 0.0)
        y = np.where(hit, res / np.where(hit, dn, 1.0), 0.0)
        scale = np.sqrt(qw / max((res ** 2).sum() / max(hit.sum(), 1), 1e-12))
        assert np.array_equal(x[R:][hit], xb[hit]) and np.all(x[R:][~hit] == 0)
        assert np.all(t[R:, 0] == 0) and np.all(m[R:, 0] == 0)
        # the kernel forms the residual in FP32: a few roundings of the terms it subtracts
        tol_y = 4 * 2.0 ** -24 * (np.abs(u_plain) + np.abs(u_off) + np.abs(sc.h * dudn) + np.abs(dt)) \
            / np.where(hit, np.abs(dn), 1.0) + 1e-6 * np.abs(y)
        assert np.all(np.abs(t[R:, 1] - y) <= tol_y), (np.abs(t[R:, 1] - y) / tol_y).max()
        assert np.allclose(m[R:, 1], scale * np.abs(dn) * hit, rtol=1e-4, atol=0)
        assert hit.sum() > 0.1 * R
