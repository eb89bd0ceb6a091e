"""Exact solutions on a disk / ball, used to pin the oracle (test infrastructure).

Each u solves  -Lap u + sigma u = f  with Dirichlet data (the source sign that
Algorithm 1 uses), and each du/dtheta solves the differential BVP of
Eq. (bvp_deriv):  (Lap - sigma) udot = 0,  udot = gdot - V_n du/dn  on the
boundary.  For a disk of radius R with r(t) = R + sum a_m cos mt + b_m sin mt
at a = b = 0, the normal velocity is V_n = 1 for R, cos mt for a_m and sin mt
for b_m, and the motion is purely radial.  kappa = sqrt(sigma).
"""
from __future__ import annotations

import numpy as np
from scipy.special import iv


def polar(x):
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return np.hypot(x[:, 0], x[:, 1]), np.arctan2(x[:, 1], x[:, 0])


def disk_screened_const(x, R: float, sigma: float, g: float = 1.0, f: float = 0.0, n_modes: int = 8):
    """Disk, constant data g, constant source f.  Returns u and du/dtheta for
    theta = [R, a_1..a_M, b_1..b_M].
      sigma > 0: u = f/s + (g - f/s) I0(k r)/I0(k R)
      sigma = 0: u = g + f (R^2 - r^2)/4
    Boundary value of udot: -V_n du/dn(R) with du/dn = (g - f/s) k I1(kR)/I0(kR)
    (sigma > 0) or -f R/2 (sigma = 0); each Fourier mode extends harmonically
    (I_m(kr)/I_m(kR) or (r/R)^m)."""
    r, th = polar(x)
    M = n_modes
    out = np.zeros((r.size, 1 + 2 * M))
    if sigma > 0:
        k = np.sqrt(sigma)
        c = g - f / sigma
        u = f / sigma + c * iv(0, k * r) / iv(0, k * R)
        dudn = c * k * iv(1, k * R) / iv(0, k * R)
        ext = [iv(m, k * r) / iv(m, k * R) for m in range(M + 1)]
    else:
        u = g + f * (R * R - r * r) / 4.0
        dudn = -f * R / 2.0
        ext = [(r / R) ** m for m in range(M + 1)]
    out[:, 0] = -dudn * ext[0]
    for m in range(1, M + 1):
        out[:, m] = -dudn * ext[m] * np.cos(m * th)
        out[:, M + m] = -dudn * ext[m] * np.sin(m * th)
    return u, out


def disk_mapped_cos(x, R: float, n_modes: int = 8):
    """Disk, sigma = 0, mapped data g(t) = cos t (fixed on the reference):
    u = x / R.  du/dn = cos t / R, so udot = -V_n cos t / R on the boundary:
      du/dR   = -x / R^2
      du/da_m = -(1/2R) [(r/R)^(m+1) cos(m+1)th + (r/R)^|m-1| cos(m-1)th]
      du/db_m = -(1/2R) [(r/R)^(m+1) sin(m+1)th + (r/R)^|m-1| sin(m-1)th]"""
    r, th = polar(x)
    M = n_modes
    u = r * np.cos(th) / R
    out = np.zeros((r.size, 1 + 2 * M))
    out[:, 0] = -r * np.cos(th) / R ** 2
    for m in range(1, M + 1):
        a = (r / R) ** (m + 1)
        b = (r / R) ** abs(m - 1)
        out[:, m] = -(a * np.cos((m + 1) * th) + b * np.cos((m - 1) * th)) / (2 * R)
        out[:, M + m] = -(a * np.sin((m + 1) * th) + b * np.sin((m - 1) * th)) / (2 * R)
    return u, out


def disk_mapped_linear(x, R: float, c: float, s: float, n_modes: int = 8):
    """Disk, sigma = 0, mapped data g(t) = c cos t + s sin t whose two
    coefficients are themselves parameters (Eq. boundary_deriv_mapped with a
    nonzero data derivative): theta = [R, a_1..a_M, b_1..b_M, c, s].
    u = (c x + s y) / R is harmonic with these boundary values, so
      du/dc = x / R,  du/ds = y / R  (the data term alone: V_n = 0 for them),
      du/dR = -(c x + s y) / R^2,
    and a_m, b_m move the boundary by V_n = cos mt, sin mt, giving the boundary
    value -V_n du/dn = -V_n (c cos t + s sin t) / R extended harmonically:
      du/da_m = -(1/2R) [c (p cos(m+1)th + q cos(m-1)th) + s (p sin(m+1)th - q sin(m-1)th)]
      du/db_m = -(1/2R) [c (p sin(m+1)th + q sin(m-1)th) + s (q cos(m-1)th - p cos(m+1)th)]
    with p = (r/R)^(m+1), q = (r/R)^|m-1|."""
    r, th = polar(x)
    M = n_modes
    u = r * (c * np.cos(th) + s * np.sin(th)) / R
    out = np.zeros((r.size, 1 + 2 * M + 2))
    out[:, 0] = -u / R
    for m in range(1, M + 1):
        p = (r / R) ** (m + 1)
        q = (r / R) ** abs(m - 1)
        out[:, m] = -(c * (p * np.cos((m + 1) * th) + q * np.cos((m - 1) * th))
                      + s * (p * np.sin((m + 1) * th) - q * np.sin((m - 1) * th))) / (2 * R)
        out[:, M + m] = -(c * (p * np.sin((m + 1) * th) + q * np.sin((m - 1) * th))
                          + s * (q * np.cos((m - 1) * th) - p * np.cos((m + 1) * th))) / (2 * R)
    out[:, 2 * M + 1] = r * np.cos(th) / R
    out[:, 2 * M + 2] = r * np.sin(th) / R
    return u, out


def harmonic_field(x, field):
    """u = g for restricted data g = c0 + c.x + x^T A x with trace(A) = 0, sigma = 0,
    f = 0, on any domain; du/dtheta = 0 for every shape parameter."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    X = np.zeros((x.shape[0], 3))
    X[:, :x.shape[1]] = x
    c0, c, A6 = field[0], np.asarray(field[1:4]), np.asarray(field[4:10])
    A = np.array([[A6[0], A6[3], A6[4]], [A6[3], A6[1], A6[5]], [A6[4], A6[5], A6[2]]])
    return c0 + X @ c + np.einsum("ni,ij,nj->n", X, A, X)


def ball_screened_const(x, R: float, sigma: float, g: float = 1.0, f: float = 0.0):
    """Ball of radius R in 3D, constant data g and source f; theta = [R].
      sigma > 0: u = f/s + (g - f/s) R sinh(k r) / (r sinh(k R)),
                 du/dR = (g - f/s) R sinh(kr)/(r sinh kR) (1/R - k coth kR)
      sigma = 0: u = g + f (R^2 - r^2)/6,  du/dR = f R / 3"""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r = np.linalg.norm(x, axis=1)
    if sigma > 0:
        k = np.sqrt(sigma)
        c = g - f / sigma
        rs = np.where(r > 1e-12, r, 1e-12)
        shape = np.where(r > 1e-12, R * np.sinh(k * rs) / (rs * np.sinh(k * R)), k * R / np.sinh(k * R))
        u = f / sigma + c * shape
        dudR = c * shape * (1.0 / R - k / np.tanh(k * R))
    else:
        u = g + f * (R * R - r * r) / 6.0
        dudR = np.full_like(r, f * R / 3.0)
    return u, dudR[:, None]


def expected_exit_weight(dim: int, sigma: float, d: float) -> float:
    """E over a uniform ball point of |B(d)| G_d(.): the solution at the centre of
    -Lap w + sigma w = 1, w = 0 on the sphere, i.e. (1 - alpha)/sigma, or
    d^2 / (2 dim) for sigma = 0."""
    if sigma <= 0:
        return d * d / (2.0 * dim)
    k = np.sqrt(sigma) * d
    alpha = 1.0 / iv(0, k) if dim == 2 else k / np.sinh(k)
    return (1.0 - alpha) / sigma


# ----------------------------------------------- mixed Dirichlet-Neumann boundaries
def quarter_disk(x, data: str):
    """Quarter disk, Dirichlet arc r = R, reflecting Neumann radii on the axes,
    sigma = 0, R = 1: u = x^2 - y^2 (harmonic, zero normal derivative on both
    axes).  theta = [R] scales the domain: for field data g = x^2 - y^2 the
    solution does not change (du/dR = 0); for mapped data g = cos 2t,
    u = (r/R)^2 cos 2 phi, du/dR = -2 (x^2 - y^2)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    u = x[:, 0] ** 2 - x[:, 1] ** 2
    du = np.zeros_like(u) if data == "field" else -2.0 * u
    return u, du[:, None]


def strip(x, sigma: float, f: float = 0.0, g: float = 1.0):
    """Rectangle with Dirichlet sides x = -1 and x = L (data g) and reflecting
    Neumann top and bottom: u depends on x alone, -u'' + sigma u = f.
      sigma > 0, f = 0: u = g cosh(k (x - c)) / cosh(k (L - c)), c = (L - 1)/2,
                        du/dL = -(g k / 2) sinh(k (x + 1)) / cosh(k)^2 at L = 1
      sigma = 0:        u = g + f (x + 1)(L - x) / 2, du/dL = f (x + 1) / 2."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))[:, 0]
    if sigma > 0:
        if f != 0:
            raise ValueError("strip: sigma > 0 with a source is not tabulated")
        k = np.sqrt(sigma)
        u = g * np.cosh(k * x) / np.cosh(k)
        du = -g * 0.5 * k * np.sinh(k * (x + 1)) / np.cosh(k) ** 2
    else:
        u = g + f * (x + 1) * (1 - x) / 2
        du = f * (x + 1) / 2
    return u, du[:, None]


def slit_sqrt(x):
    """Unit disk cut along [0, 1) x {0} (reflecting on both sides), sigma = 0,
    Dirichlet data cos(t / 2) on the circle: u = sqrt(r) cos(phi / 2) with phi
    in (0, 2 pi) measured from the slit (harmonic, zero normal derivative on
    both faces of the slit, equal to the data on the circle)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r = np.hypot(x[:, 0], x[:, 1])
    phi = np.mod(np.arctan2(x[:, 1], x[:, 0]), 2 * np.pi)
    return np.sqrt(r) * np.cos(phi / 2)


def cube_linear(x, f: float = 0.0):
    """Cube with Dirichlet faces x = -1 (g = -1) and x = X (g = 1), reflecting
    Neumann elsewhere, sigma = 0, constant source f of -u'' = f: u depends on
    x alone, u = 2 (x + 1) / (X + 1) - 1 + f (x + 1) (X - x) / 2, so at X = 1
    u = x + f (1 - x^2) / 2 and du/dX = -(x + 1) / 2 + f (x + 1) / 2."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    xx = x[:, 0]
    return xx + f * (1 - xx * xx) / 2, ((xx + 1) * (f - 1) / 2)[:, None]


def cube_screened(x, sigma: float):
    """Cube with Dirichlet faces x = -1 (g = -1) and x = X (g = 1), reflecting
    Neumann elsewhere, -u'' + sigma u = 0 (k = sqrt(sigma)): u depends on x
    alone, u = (sinh(k (x + 1)) - sinh(k (X - x))) / sinh(k (X + 1)), at X = 1
    sinh(k x) / sinh(k); du/dX is its central difference in X (step 1e-6, an
    error of order 1e-12 against the exact derivative)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    k = np.sqrt(sigma)
    xx = x[:, 0]
    u = lambda X: (np.sinh(k * (xx + 1)) - np.sinh(k * (X - xx))) / np.sinh(k * (X + 1))
    d = 1e-6
    return u(1.0), ((u(1.0 + d) - u(1.0 - d)) / (2 * d))[:, None]


def cylinder_flow(x, a: float):
    """Potential flow past a cylinder: u = x (1 + a^2 / r^2) = (r + a^2 / r) cos phi
    is harmonic where r > 0 (the radial part f = r + a^2/r has
    f'' + f'/r - f/r^2 = 0) and du/dr = f'(a) cos phi = 0 on the circle r = a:
    with a reflecting Neumann circle of radius a and Dirichlet data u on an
    outer boundary, the solution is u itself.  With the data scaled by a
    parameter c (at c = 1), du/dc = u."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r2 = x[:, 0] ** 2 + x[:, 1] ** 2
    u = x[:, 0] * (1.0 + a * a / r2)
    return u, u[:, None].copy()


def sphere_flow(x, a: float, q: float = 0.0):
    """Potential flow past a sphere: u = x (1 + a^3 / (2 r^3)) = f(r) cos(theta)
    with f = r + a^3 / (2 r^2), harmonic where r > 0 (f'' + 2 f'/r - 2 f/r^2 = 0)
    and du/dr = f'(a) cos(theta) = 0 on the sphere r = a: with a reflecting
    Neumann sphere of radius a and Dirichlet data u on an outer boundary, the
    solution is u itself.  With the data scaled by a parameter c (at c = 1),
    du/dc = u.  A source q / r (harmonic, du/dn = q / a^2 on the sphere with n
    towards the centre) adds to u with data q / a^2 on the sphere and q / r on
    the outer boundary; unscaled by c, it leaves du/dc as it was."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r3 = np.sum(x * x, axis=1) ** 1.5
    u = x[:, 0] * (1.0 + a ** 3 / (2.0 * r3))
    return u + q / np.cbrt(r3), u[:, None].copy()


def neumann_data_box(x, c: float, b: float):
    """Neumann data on the box [-1, 1]^d: the faces x = -1 and x = X (X = 1)
    Dirichlet, the others Neumann with data du/dn = 2c (n out of the box), and
    restricted Dirichlet data g = b x + c (y^2 - x^2) (2D), b x + c (y^2 + z^2 -
    2 x^2) (3D).  g is harmonic and its normal derivative on the Neumann faces
    is 2c, so u = g in the whole box whatever X is: du/dX = 0."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    if x.shape[1] == 2:
        u = b * x[:, 0] + c * (x[:, 1] ** 2 - x[:, 0] ** 2)
    else:
        u = b * x[:, 0] + c * (x[:, 1] ** 2 + x[:, 2] ** 2 - 2 * x[:, 0] ** 2)
    return u, np.zeros((len(u), 1))


def screened_neumann_data_box(x, k: float, s: float):
    """-Lap u + k^2 u = 0 on [-1, X] x [-1, 1] with Neumann data du/dn =
    k sinh(k) on y = -1, 1 and Dirichlet data g = cosh(k y) - s sinh(k) on
    x = -1 and cosh(k y) + s sinh(k) on x = X, each carried by its side's
    vertices as X moves: u = cosh(k y) + w(x) with w'' = k^2 w, w(-1) = -S,
    w(X) = S (S = s sinh k), i.e. w = S (sinh(k (x + 1)) - sinh(k (X - x))) /
    sinh(k (X + 1)), at X = 1 s sinh(k x).  du/dX is the central difference of
    w in X (step 1e-6)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    S = s * np.sinh(k)
    xx = x[:, 0]
    w = lambda X: S * (np.sinh(k * (xx + 1)) - np.sinh(k * (X - xx))) / np.sinh(k * (X + 1))
    d = 1e-6
    return np.cosh(k * x[:, 1]) + w(1.0), ((w(1.0 + d) - w(1.0 - d)) / (2 * d))[:, None]


def annulus_log(x, a: float, b: float):
    """u = a + b log r on r_in < r < 1: the outer circle carries Dirichlet
    data a, the inner circle Neumann data du/dn = -b / r_in (n out of the
    domain points to the centre)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return a + b * np.log(np.hypot(x[:, 0], x[:, 1]))
