"""The ball-gradient du/dn estimator (Eq. dudn_mc_estimate) in the oracle.

Pins:
  * the factor F of grad u(c) = F E[n_y u(y)] against quadrature of exact
    solutions on the circle / sphere: plane waves e^{k x.e} of
    -Lap u + k^2 u = 0 and the harmonic e^x cos y at sigma = 0;
  * the estimator's mean on the screened disk equals the closed-form radial
    derivative at the offset point (it estimates grad u there, not at xbar);
  * for u = x its mean is n_x exactly while its variance is not zero.
"""
import numpy as np
import pytest

import oracle
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle


def _sphere_mean(dim, R, c, u):
    """E[n_y u(c + R n_y)] for y uniform on the sphere (quadrature)."""
    if dim == 2:
        t = (np.arange(4096) + 0.5) * (2 * np.pi / 4096)
        n = np.stack([np.cos(t), np.sin(t)], 1)
        return (n * u(c + R * n)[:, None]).mean(0)
    z, wz = np.polynomial.legendre.leggauss(64)
    ph = (np.arange(128) + 0.5) * (2 * np.pi / 128)
    Z, PH = np.meshgrid(z, ph, indexing="ij")
    W = np.repeat(wz[:, None], 128, 1) / (2 * 128)
    st = np.sqrt(1 - Z ** 2)
    n = np.stack([st * np.cos(PH), st * np.sin(PH), Z], -1).reshape(-1, 3)
    return (n * (u(c + R * n) * W.reshape(-1))[:, None]).sum(0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.25, 4.0, 40.0])
def test_factor_recovers_plane_wave_gradients(dim, sigma):
    k = np.sqrt(sigma)
    e = np.array([0.6, 0.8, 0.0][:dim]) if dim == 2 else np.array([2.0, -1.0, 2.0]) / 3.0
    c = np.array([0.3, -0.2, 0.1][:dim])
    u = lambda x: np.exp(k * (x @ e))
    for R in (0.01, 0.3, 1.5):
        got = oracle.gradient_factor(dim, sigma, R) * _sphere_mean(dim, R, c, u)
        want = k * np.exp(k * (c @ e)) * e
        assert np.allclose(got, want, rtol=1e-9, atol=1e-12), (R, got, want)


def test_factor_recovers_a_harmonic_gradient():
    c = np.array([0.2, 0.4])
    u = lambda x: np.exp(x[:, 0]) * np.cos(x[:, 1])
    want = np.array([np.exp(0.2) * np.cos(0.4), -np.exp(0.2) * np.sin(0.4)])
    for R in (0.05, 0.7):
        got = oracle.gradient_factor(2, 0.0, R) * _sphere_mean(2, R, c, u)
        assert np.allclose(got, want, rtol=1e-9)


def _hits(sc, W, mode):
    o = oracle.run_walks(to_oracle(sc, dudn_mode=mode), sc.query, W, differential=True)
    hit = o["elem"] >= 0
    return o, hit


def test_mean_is_the_gradient_at_the_offset_point():
    sc = scenes.disk_scene("screened_1", n_query=16)
    o, hit = _hits(sc, 2048, 1)
    from scipy.special import iv
    k, R = 2.0, 1.0
    want = k * iv(1, k * (R - sc.h)) / iv(0, k * R)       # d/dr of I0(k r) / I0(k R) at r = R - h
    d = o["dudn"][hit]
    se = d.std(ddof=1) / np.sqrt(d.size)
    # the 128-gon is inside the disk by its sagitta (3e-4): a few 1e-3 of bias at most
    assert abs(d.mean() - want) < 4.5 * se + 5e-3 * want, (d.mean(), want, se)
    # the backward difference estimates (u(xbar) - u(x_off)) / h instead: both near want
    o2, hit2 = _hits(sc, 2048, 0)
    assert abs(o2["dudn"][hit2].mean() - want) < 0.05 * want


def test_linear_solution_gives_the_exact_mean():
    sc = scenes.disk_scene("laplace_x", n_query=16)
    o, hit = _hits(sc, 1024, 1)
    r = o["dudn"][hit] - o["normal"][hit, 0]
    assert r.std() > 0.1
    assert abs(r.mean()) < 4.5 * r.std(ddof=1) / np.sqrt(r.size)
