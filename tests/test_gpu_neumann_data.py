"""Walks on stars with Neumann data on the GPU (Sec. 3.4, Eq. mixed_bvp with
Robin coefficient 0 and data h = du/dn) against the FP64 oracle, through the C
ABI (dwos_set_neumann_data).

* Per-walk replays of the same Philox walks (the data sample draws its element
  by per-element keys, so the pick does not depend on the tree's order): on
  walks whose branch matches, nearly every u and udot lies within the tight
  per-walk bound, and per point the mean difference over those walks is a
  tenth of the estimator's error bar or less.  A sample whose point lands
  close to the walk (G_R is singular there) carries the FP32 walk's position
  drift, relative to the distance, into u: those walks (about 1 % on the
  cube, 4 % on the annulus, whose walks sit on a polygonal circle) are what
  the fraction allows.
* Per-point means against the closed forms of the square and cube with
  Neumann data (u and du/dX = 0), the screened square and the annulus; the
  thermal design with data varying from element to element replays too.
* The entry point: zero data runs the reflecting walks bit for bit, data set
  before the Neumann flags applies, and non-finite data is refused.
"""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_2405_12964_gb300 import scenes
from tests.test_gpu_parity import branch_match, gpu_udot, run_pair, u_drift_allowance

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


def _replay(Solver, sc, W, differential=True, u_scale=0.0, min_tight=0.98):
    s, g, o = run_pair(Solver, sc, W, differential=differential)
    n = sc.query.shape[0]
    same = branch_match(sc, g, o, differential)
    assert 1 - same.mean() <= 0.03, 1 - same.mean()
    dirichlet = np.nonzero(sc.neumann == 0)[0]
    ended = g["rec"]["elem"] >= 0
    assert np.isin(g["rec"]["elem"][ended], dirichlet).all()
    pt = np.repeat(np.arange(n), W)[same]
    cnt = np.maximum(np.bincount(pt, minlength=n), 1)
    ug, uo = g["rec"]["u"].astype(np.float64), o["u_hat"]
    err = np.abs(ug - uo)[same]
    tol = 1e-4 * (np.abs(uo[same]) + u_scale) + 1e-5 + u_drift_allowance(sc, g["rec"], o)[same]
    frac = (err <= tol).mean()
    d = np.bincount(pt, weights=(ug - uo)[same], minlength=n) / cnt
    se = uo.reshape(n, W).std(axis=1) / np.sqrt(W)
    print("%s: %.4f same branch, %.4f within the tight bound, max |mean diff| / SE %.3g"
          % (sc.name, same.mean(), frac, np.max(np.abs(d) / (se + 1e-30))))
    assert frac >= min_tight, frac
    assert np.all(np.abs(d) <= 0.1 * se + 1e-4 * (np.abs(uo.reshape(n, W).mean(axis=1)) + u_scale)), (d, se)
    if differential and sc.n_param:
        P = sc.n_param
        dg, do = gpu_udot(sc, g["rec"]), o["udot"]
        e2 = np.abs(dg - do)[same]
        frac2 = (e2 <= 1e-3 * (1 + np.abs(do[same]))).mean()
        dd = np.stack([np.bincount(pt, weights=(dg - do)[same, j], minlength=n) / cnt for j in range(P)], 1)
        se2 = do.reshape(n, W, P).std(axis=1) / np.sqrt(W)
        print("%s: udot %.4f within the tight bound, max |mean diff| / SE %.3g"
              % (sc.name, frac2, np.max(np.abs(dd) / (se2 + 1e-30))))
        assert frac2 >= min_tight, frac2
        assert np.all(np.abs(dd) <= 0.1 * se2 + 1e-3 * (1 + np.abs(do.reshape(n, W, P).mean(axis=1)))), (dd, se2)
    return s, g, o, same


def _eval(s, sc, W, grad=True):
    out = s.eval(sc.query, W, grad=grad)
    r = {"u": out["u"].cpu().numpy(), "u_se": out["u_se"].cpu().numpy()}
    if grad:
        r["du"], r["du_se"] = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    return r


def _close(m, se, exact, rel, ab, floor=False):
    if floor:
        se = np.maximum(se, np.median(se, axis=0, keepdims=True))
    assert np.all(np.abs(m - exact) <= 4.5 * se + rel * np.abs(exact) + ab), (np.abs(m - exact) / se, m, exact)


@pytest.mark.parametrize("dim", [2, 3])
def test_box_with_neumann_data_replay_and_closed_form(Solver, dim):
    sc = scenes.neumann_data_box_scene(dim, c=0.5, b=0.3, n_query=6)
    face = sc.query[:2].copy()
    face[:, 1] = [-1.0, 1.0]                               # on the Neumann faces y = -1, 1
    sc.query = np.concatenate([sc.query, face])
    s, g, o, same = _replay(Solver, sc, 64, u_scale=1.0, min_tight=0.98 if dim == 2 else 0.97)
    r = _eval(s, sc, 8192)
    u, du = cf.neumann_data_box(sc.query, 0.5, 0.3)
    _close(r["u"], r["u_se"], u, 0.0, 4e-3)
    _close(r["du"], r["du_se"], du, 0.0, 0.02, floor=True)


def test_screened_square_with_neumann_data_replay_and_closed_form(Solver):
    sc = scenes.screened_neumann_data_box_scene(k=1.5, s=0.5, n_query=8)
    s, g, o, same = _replay(Solver, sc, 64, u_scale=2.0)
    assert (o["kind"][:, 0] == oracle.KIND_ROULETTE).any()
    r = _eval(s, sc, 8192)
    u, du = cf.screened_neumann_data_box(sc.query, 1.5, 0.5)
    _close(r["u"], r["u_se"], u, 3e-3, 2e-3)
    _close(r["du"], r["du_se"], du, 0.08, 0.02, floor=True)


def test_annulus_with_neumann_data_replay_and_closed_form(Solver):
    sc = scenes.annulus_neumann_data_scene(n_query=8)
    # walks on the polygonal circle take short steps (R reaches the next vertex, a silhouette
    # point) with samples close to the walk: more of them carry the drift
    s, g, o, same = _replay(Solver, sc, 64, differential=False, u_scale=1.0, min_tight=0.9)
    r = _eval(s, sc, 8192, grad=False)
    _close(r["u"], r["u_se"], cf.annulus_log(sc.query, 1.0, 0.5), 0.0, 3e-3)


def test_thermal_design_with_varying_neumann_data_replays(Solver):
    # data that changes from element to element on the slab (and its ends), query points on the
    # slab's underside: the element draw, the data lookup and the share 1/2 at the start
    sc = scenes.thermal_scene(n_query=8)
    idx = np.arange(len(sc.elem))
    sc.neumann_h = np.where(sc.neumann == 1, 0.5 + 0.4 * np.sin(0.7 * idx), 0.0)
    _replay(Solver, sc, 64, u_scale=1.0, min_tight=0.95)


def test_neumann_data_entry_point(Solver):
    import copy
    sc = scenes.neumann_data_box_scene(2, c=0.5, b=0.3, n_query=4)
    bare = copy.copy(sc)
    bare.neumann_h = None

    def records(s):
        return s.walk_records(sc.query, 32, walk_id_base=0, differential=True)["rec"]

    plain = Solver(0)
    plain.load_scene(bare)
    zero = Solver(0)
    zero.load_scene(bare)
    zero.set_neumann_data(np.zeros(len(sc.elem)))
    a = records(plain)
    assert np.array_equal(a.view(np.uint8), records(zero).view(np.uint8))
    loaded = Solver(0)
    loaded.load_scene(sc)
    c = records(loaded)
    assert not np.array_equal(a["u"], c["u"])
    # data given before the Neumann flags applies once they are set
    first = Solver(0)
    nf = copy.copy(bare)
    nf.neumann = None
    first.load_scene(nf)
    first.set_neumann_data(sc.neumann_h)
    first.set_neumann(sc.neumann)
    assert np.array_equal(c.view(np.uint8), records(first).view(np.uint8))
    # a new boundary clears it
    again = Solver(0)
    again.load_scene(sc)
    again.load_scene(bare)
    assert np.array_equal(a.view(np.uint8), records(again).view(np.uint8))
    bad = sc.neumann_h.copy()
    bad[3] = np.nan
    with pytest.raises(Exception):
        loaded.set_neumann_data(bad)
