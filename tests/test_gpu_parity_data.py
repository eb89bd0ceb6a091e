"""GPU parity for the boundary-data derivative, the 2D source term and the
ball weights behind it (through the C ABI, against the FP64 oracle).

* Eq. (boundary_deriv_mapped) with a nonzero data derivative dg_v/dtheta: the
  per-walk records, the forward-mode means and the reverse-mode (U-statistic
  gradient, VJP) sums against the oracle on the same Philox walks, and the
  disk's closed form u = (c x + s y)/R, du/dc = x/R, du/ds = y/R.
* The source estimate of Algorithm 1 in 2D (Sec. 3.3, Eq. wos): per-walk replay
  with f != 0 at sigma = 0 (the log branch) and sigma = 3 (the K0 / I0 branch),
  and the disk's closed form u = f/s + (g - f/s) I0(kr)/I0(kR).
* The device's ball weights |B| G and alpha, and its K0, against the oracle's
  FP64 definitions (std::cyl_bessel_k / i), element by element.
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


# ------------------------------------------------------------------ special functions
def test_bessel_k0_matches_library_routine(Solver):
    # Tolerance: the A&S 9.8.5 polynomial is within 1e-8 absolute for x <= 2 and
    # 9.8.6 within 1.9e-7 on x^(1/2) e^x K0 (>= 1.19 for x >= 2: 1.6e-7 relative);
    # FP32 evaluation adds about a dozen roundings (Horner steps, exp, rsqrt, log,
    # CUDA's I0 at <= 6 ulp): under 8e-7 relative.  Both sides see the same FP32 x.
    s = Solver(0)
    x = np.concatenate([np.geomspace(1e-4, 80.0, 3000), [2.0, np.nextafter(2.0, 3.0)]]).astype(np.float32)
    got = s.bessel_k0(x).astype(np.float64)
    want = np.array([oracle.bessel_k0(float(v)) for v in x])
    assert np.allclose(want, k0(x.astype(np.float64)), rtol=1e-13)       # the oracle's routine is the textbook K0
    err = np.abs(got - want)
    tol = 1e-6 * want + 1e-8
    assert np.all(err <= tol), (x[np.argmax(err / tol)], (err / tol).max())
    print("K0: max relative error %.2e" % (err / want).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_ball_weights_match_oracle(Solver, dim):
    # The source factor |B(d)| G_d(r) and the recursive weight alpha as the walk
    # kernel evaluates them, against the oracle's FP64 formulas at the same FP32
    # inputs.  Tolerance per value: the functions' own FP32 error (a few ulp each,
    # 2e-6 relative of the magnitude M of the terms that are summed) plus the
    # rounding of the arguments (k = sqrtf(sigma), kd, kr: <= 4 roundings, 2.4e-7
    # relative) amplified by the functions' log-derivatives, bounded by 1 + kd + kr.
    s = Solver(0)
    rng = np.random.default_rng(11)
    for sigma in (0.0, 0.3, 4.0, 100.0, 2500.0):
        for d in (1e-3, 0.02, 0.3, 1.0, 2.0):
            u = rng.uniform(0.0, 1.0, 200).astype(np.float32)
            u = np.clip(u, 1e-6, 1 - 1e-6).astype(np.float32)
            dd = np.full(u.shape, d, np.float32)
            src, alpha = s.ball_weights(dim, sigma, dd, u)
            d64 = float(np.float32(d))
            rho = u.astype(np.float64) ** (1.0 / dim)
            ref_src = np.array([oracle.source_weight(dim, float(np.float32(sigma)), d64, r) for r in rho])
            ref_alpha = oracle.alpha(dim, float(np.float32(sigma)), d64)
            k = np.sqrt(float(np.float32(sigma)))
            kd, kr = k * d64, k * d64 * rho
            if dim == 2:
                if k > 0:
                    M = 0.5 * d64 ** 2 * (k0(kr) + (k0(kd) * i0(kr) / i0(kd) if kd < 80 else 0.0))
                else:
                    M = 0.25 * d64 ** 2 * np.abs(np.log(u.astype(np.float64))) + 0.25 * d64 ** 2 * 1e-6
            else:
                M = d64 ** 2 / 3.0 / rho * (1.0 + 1e-6)
            A = 1.0 + kd + kr
            tol = M * (2e-6 + 2.4e-7 * A) + 1e-37
            err = np.abs(src.astype(np.float64) - ref_src)
            assert np.all(err <= tol), (sigma, d, (err / tol).max())
            tol_a = ref_alpha * (1e-6 + 2.4e-7 * (1.0 + kd)) + 1e-37
            assert np.all(np.abs(alpha.astype(np.float64) - ref_alpha) <= tol_a), (sigma, d, alpha[0], ref_alpha)


# ------------------------------------------------------------------ 2D source walks
@pytest.mark.parametrize("sigma", [0.0, 3.0])
def test_2d_source_walks_replay_and_closed_form(Solver, sigma):
    sc = scenes.disk_scene("screened_1", n_query=16)
    sc.sigma, sc.f = sigma, 2.0
    s, g, o = run_pair(Solver, sc, 128)
    same = check_walks(sc, g, o)
    # the source sum is the bulk of u here (f (R^2 - r^2)/4 at sigma = 0)
    assert np.mean(np.abs(o["u_hat"][same] - 1.0)) > 0.05
    out = s.eval(sc.query, 4096, grad=True)
    u, use = out["u"].cpu().numpy(), out["u_se"].cpu().numpy()
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    ue, due = cf.disk_screened_const(sc.query, 1.0, sigma, g=1.0, f=2.0)
    assert np.all(np.abs(u - ue) <= 4.5 * use + 3e-3 * np.abs(ue) + 1e-3), np.abs(u - ue) / use
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))[:, :3]
    assert np.all(np.abs(du[:, :3] - due[:, :3]) <= 4.5 * dse_ref + 0.08 * np.abs(due[:, :3]) + 0.01)


# ------------------------------------------------------------------ boundary-data derivative
def test_data_parameter_derivative_on_the_disk(Solver):
    sc = scenes.disk_scene("mapped_data", n_query=16)
    s, g, o = run_pair(Solver, sc, 128)
    check_walks(sc, g, o, u_scale=np.abs(sc.g_vert).max())
    out = s.eval(sc.query, 8192, grad=True)
    du, dse = out["du"].cpu().numpy(), out["du_se"].cpu().numpy()
    _, due = cf.disk_mapped_linear(sc.query, 1.0, sc.meta["c"], sc.meta["s"])
    # the data columns (c, s): no 1/h noise, bias from the polygon's interpolation only
    assert np.all(np.abs(du[:, -2:] - due[:, -2:]) <= 4.5 * dse[:, -2:] + 4e-3 * np.abs(due[:, -2:]) + 1e-3)
    dse_ref = np.maximum(dse, np.median(dse, axis=0, keepdims=True))
    assert np.all(np.abs(du - due) <= 4.5 * dse_ref + 0.08 * np.abs(due) + 0.01)


def _star_with_data_derivative(n_query=16, walks=64, seed=21):
    sc = scenes.star_box_scene(n_seg=1024, n_query=n_query, walks=walks)
    rng = np.random.default_rng(seed)
    # every parameter also moves the data: random dg_v/dtheta on the star's vertices and
    # on two box corners (the box moves nowhere, so only its data term reaches theta)
    dg = np.zeros((sc.vert.shape[0], sc.n_param))
    dg[4:] = rng.normal(0.0, 0.5, size=(sc.vert.shape[0] - 4, sc.n_param))
    dg[[0, 2]] = rng.normal(0.0, 0.5, size=(2, sc.n_param))
    sc.dg_vert = dg
    return sc


def test_data_parameter_derivative_per_walk_on_the_star(Solver):
    sc = _star_with_data_derivative(n_query=24)
    s, g, o = run_pair(Solver, sc, 32)
    same = check_walks(sc, g, o)
    # the data term is a large part of every shell hit's derivative
    hit = same & (o["elem"] >= 0)
    assert np.abs(o["udot"][hit]).mean() > 0.1


def test_data_parameter_derivative_reverse_mode(Solver):
    sc = _star_with_data_derivative()
    s = Solver(0)
    s.load_scene(sc)
    o = oracle.run_walks(to_oracle(sc), sc.query, sc.walks, differential=True)
    n = sc.query.shape[0]
    loss, gr = (t.cpu().numpy() for t in s.grad_l2(sc.query, sc.u_ref, sc.walks))
    go = est.grad_l2_ustat(o["u_hat"], o["udot"], sc.u_ref, n, sc.walks, 8)
    scale = np.abs(go).max()
    assert np.allclose(gr, go, rtol=2e-3, atol=2e-3 * scale), np.abs(gr - go).max() / scale
    assert abs(loss[0] - est.loss_l2(o["u_hat"], sc.u_ref, n, sc.walks)) <= 1e-4 * abs(loss[0]) + 1e-7
    w = np.linspace(-1.0, 1.0, n)
    gv = s.vjp(sc.query, w, sc.walks, walk_id_base=0).cpu().numpy()
    vo = est.vjp(o["udot"], w, n, sc.walks)
    assert np.allclose(gv, vo, rtol=2e-3, atol=2e-3 * np.abs(vo).max())
    # without the data derivative the gradient is a different vector: the dg term is live
    s2 = Solver(0)
    s2.load_scene(sc)
    s2.set_dirichlet_mapped(sc.g_vert)
    g0 = s2.grad_l2(sc.query, sc.u_ref, sc.walks)[1].cpu().numpy()
    assert np.abs(g0 - gr).max() > 0.2 * scale
