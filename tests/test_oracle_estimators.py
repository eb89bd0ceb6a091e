"""Pins for the product estimators of Sec. 4.3 (Eqs. uncorrelated_product,
correlated_product, ustatistics_unrolled, ustatistics)."""
import numpy as np

from oracle import estimators as est


def test_ustat_linear_form_equals_pairwise_double_sum():
    rng = np.random.default_rng(0)
    for n in [2, 3, 8, 17]:
        u = rng.normal(size=n)
        ud = rng.normal(size=(n, 5))
        pair = np.zeros(5)
        for m in range(n):
            for mp in range(n):
                if m != mp:
                    pair += u[m] * ud[mp]
        pair /= n * (n - 1)
        assert np.allclose(est.ustat_product(u, ud), pair, rtol=1e-12, atol=1e-14)


def test_ustat_is_unbiased_and_correlated_product_is_not():
    # u_m = X_m, udot_m = X_m + Y_m with X ~ N(mu, 1), Y ~ N(nu, 1):
    # E[u] E[udot] = mu (mu + nu); the correlated product adds Var(X)/n.
    rng = np.random.default_rng(1)
    mu, nu, n, reps = 0.7, -0.2, 8, 40000
    X = rng.normal(mu, 1.0, size=(reps, n))
    Y = rng.normal(nu, 1.0, size=(reps, n))
    ud = (X + Y)[..., None]
    us = np.array([est.ustat_product(X[r], ud[r])[0] for r in range(reps)])
    cor = (X.mean(1) * (X + Y).mean(1))
    target = mu * (mu + nu)
    assert abs(us.mean() - target) < 4 * us.std() / np.sqrt(reps)
    assert abs(cor.mean() - (target + 1.0 / n)) < 4 * cor.std() / np.sqrt(reps)
    assert abs(cor.mean() - target) > 8 * cor.std() / np.sqrt(reps)


def test_grad_l2_ustat_per_batch_definition():
    rng = np.random.default_rng(2)
    P, W, B, N = 3, 16, 8, 4
    u = rng.normal(size=P * W)
    ud = rng.normal(size=(P * W, N))
    ur = rng.normal(size=P)
    got = est.grad_l2_ustat(u, ud, ur, P, W, B)
    want = np.zeros(N)
    for p in range(P):
        acc = np.zeros(N)
        for b in range(W // B):
            rows = slice(p * W + b * B, p * W + (b + 1) * B)
            uu, dd = u[rows], ud[rows]
            pair = sum(uu[m] * dd[k] for m in range(B) for k in range(B) if m != k) / (B * (B - 1))
            acc += pair - ur[p] * dd.mean(0)
        want += acc / (W // B)
    assert np.allclose(got, want, rtol=1e-12)


def test_uncorrelated_and_vjp_definitions():
    rng = np.random.default_rng(3)
    P, W, N = 2, 10, 3
    u = rng.normal(size=P * W)
    ud = rng.normal(size=(P * W, N))
    ur = rng.normal(size=P)
    g = est.grad_l2_uncorrelated(u, ud, ur, P, W)
    want = sum((u[p * W:p * W + 5].mean() - ur[p]) * ud[p * W + 5:p * W + 10].mean(0) for p in range(P))
    assert np.allclose(g, want)
    w = rng.normal(size=P)
    assert np.allclose(est.vjp(ud, w, P, W), sum(w[p] * ud[p * W:(p + 1) * W].mean(0) for p in range(P)))


def test_small_cases_worked_by_hand():
    # one point, two walks: u = (1, 3), udot = (2, 4), target 1, all values worked out by hand
    u = np.array([1.0, 3.0])
    ud = np.array([[2.0], [4.0]])
    # sample mean 2; sample standard deviation (n - 1 = 1) sqrt(2); standard error sqrt(2) / sqrt(2) = 1
    m, se = est.point_mean_se(u, 1, 2)
    assert m[0] == 2.0 and abs(se[0] - 1.0) < 1e-15
    # loss: 1/2 (2 - 1)^2 = 1/2
    assert est.loss_l2(u, [1.0], 1, 2) == 0.5
    # correlated product: (mean u - target) mean udot = (2 - 1) * 3 = 3
    assert est.grad_l2_correlated(u, ud, [1.0], 1, 2)[0] == 3.0
    # uncorrelated product: u from walk 1, udot from walk 2: (1 - 1) * 4 = 0; with target 0: 1 * 4
    assert est.grad_l2_uncorrelated(u, ud, [1.0], 1, 2)[0] == 0.0
    assert est.grad_l2_uncorrelated(u, ud, [0.0], 1, 2)[0] == 4.0
    # U-statistic, one batch of B = 2: (udot_1 u_2 + udot_2 u_1) / 2 - target mean udot = (6 + 4) / 2 - 3 = 2
    assert est.grad_l2_ustat(u, ud, [1.0], 1, 2, 2)[0] == 2.0
