"""Pins for the ball Green's function G and the recursive weight alpha = P |dB|.

G and P are not printed in the paper (Sec. 3.3.1 cites WoSt App. A); the oracle
derives them from the PDE.  These tests check the oracle's functions against
facts fixed by the mathematics, not against retyped formulas: the PDE itself,
the boundary condition, the point-source singularity, the mean exit time, and
the flux identity that links P to G.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import i0

import oracle
from oracle import closed_forms as cf


def G(dim, sigma, R, r):
    """Green's function recovered from the oracle's source weight |B(R)| G(r)."""
    vol = np.pi * R * R if dim == 2 else 4.0 / 3.0 * np.pi * R ** 3
    return oracle.source_weight(dim, sigma, R, r / R) / vol


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.0, 0.7, 9.0])
def test_green_solves_screened_equation_and_vanishes_on_sphere(dim, sigma):
    R = 1.3
    for r in [0.2, 0.5, 0.9, 1.1]:
        hh = 1e-4
        g0, gp, gm = G(dim, sigma, R, r), G(dim, sigma, R, r + hh), G(dim, sigma, R, r - hh)
        d2 = (gp - 2 * g0 + gm) / hh ** 2
        d1 = (gp - gm) / (2 * hh)
        lap = d2 + (dim - 1) / r * d1            # radial Laplacian
        assert abs(-lap + sigma * g0) < 1e-5 * max(1.0, abs(d2))
    assert abs(G(dim, sigma, R, R * (1 - 1e-12))) < 1e-9


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.0, 2.0])
def test_green_has_unit_point_source(dim, sigma):
    # -Lap G = delta: flux of -grad G through a small sphere around the centre is 1
    R, r = 1.0, 1e-4
    hh = 1e-7
    dG = (G(dim, sigma, R, r + hh) - G(dim, sigma, R, r - hh)) / (2 * hh)
    area = 2 * np.pi * r if dim == 2 else 4 * np.pi * r * r
    assert abs(-dG * area - 1.0) < 1e-3


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.0, 0.5, 4.0, 25.0])
def test_alpha_is_poisson_kernel_flux_of_green(dim, sigma):
    # P = -dG/dn on the sphere; alpha = P |dB|
    R = 0.8
    hh = 1e-6
    dG = (G(dim, sigma, R, R - hh) - G(dim, sigma, R, R - 3 * hh)) / (2 * hh)
    area = 2 * np.pi * R if dim == 2 else 4 * np.pi * R * R
    alpha = -dG * area
    assert abs(alpha - oracle.alpha(dim, sigma, R)) < 2e-4


def test_alpha_special_cases():
    for dim in (2, 3):
        assert oracle.alpha(dim, 0.0, 3.0) == 1.0
        assert abs(oracle.alpha(dim, 1e-12, 1.0) - 1.0) < 1e-9
        assert oracle.alpha(dim, 100.0, 2.0) < 1e-6
    # 2D reduces to a library routine: 1 / I0(kR)
    for s, R in [(4.0, 1.0), (10.0, 0.3), (0.01, 2.0)]:
        assert abs(oracle.alpha(2, s, R) - 1.0 / i0(np.sqrt(s) * R)) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [0.0, 1.0, 10.0])
def test_mean_source_weight_is_expected_exit_time(dim, sigma):
    # E over a uniform point of the ball of |B| G = solution of -Lap w + s w = 1 at the centre
    R = 0.7
    dens = (lambda rho: 2 * rho) if dim == 2 else (lambda rho: 3 * rho * rho)
    val, _ = integrate.quad(lambda rho: oracle.source_weight(dim, sigma, R, rho) * dens(rho), 0, 1,
                            limit=200, points=[1e-6, 1e-3])
    assert abs(val - cf.expected_exit_weight(dim, sigma, R)) < 1e-7
