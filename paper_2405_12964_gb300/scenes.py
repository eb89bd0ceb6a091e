"""Seeded synthetic scenes for the walk-on-spheres workloads.

This module builds geometry and parameterisations only: polygons, star curves,
geodesic icospheres perturbed by spherical harmonics, the per-vertex parameter
Jacobians dv/dtheta of the explicit-surface parameterisation (Sec. 3.1.2), and
query points.  It contains none of the estimator's arithmetic, so that the CUDA
path and the FP64 oracle can both be fed from it.  Every array is float64 /
int32 numpy; the CUDA binding casts to float32 itself.

Scenes (all seeds fixed; geometry seed 0x2405):
  disk_scene       128-gon of radius R with radial Fourier parameters
  star_box_scene   star-shaped emitter inside the box [-1, 1]^2
  sh_sphere_scene  SH-perturbed icosphere inside the box [-2, 2]^3
  translated_star_scene  the star_box geometry with the star's position as the parameter
  mixed boundaries (a Dirichlet part and a Neumann part, reflecting unless
  the scene sets neumann_h):
  quarter_disk_scene, strip_scene, slit_disk_scene, cube_neumann_scene,
  thermal_scene (a heating wire under an insulating slab, observed on the slab)
  Neumann data (du/dn given on the Neumann part): neumann_data_box_scene,
  screened_neumann_data_box_scene, annulus_neumann_data_scene
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from math import factorial
from typing import Optional

import numpy as np

GEOMETRY_SEED = 0x2405
PHILOX_SEED = 0x12964


@dataclass
class Scene:
    """Boundary, data and PDE of one Dirichlet screened-Poisson problem.

    vert   (n_vert, dim) float64     elem  (n_elem, dim) int32
    jac    (n_vert, dim, N) float64 or None: dv/dtheta per vertex
    data   'mapped' with g_vert (n_vert,) [and dg_vert (n_vert, N)], or
           'field' with field = [c0, c(3), Axx, Ayy, Azz, Axy, Axz, Ayz]
    sigma  screening; f: constant source of -Lap u + sigma u = f
    eps    shell width; h: normal-derivative offset; K: nested walks
    query  (n_query, dim) float64; walks: walks per query point
    """
    name: str
    vert: np.ndarray
    elem: np.ndarray
    jac: Optional[np.ndarray]
    data: str = "mapped"
    g_vert: Optional[np.ndarray] = None
    dg_vert: Optional[np.ndarray] = None
    field: Optional[np.ndarray] = None
    sigma: float = 0.0
    f: float = 0.0
    eps: float = 1e-3
    h: float = 1e-2
    K: int = 1
    B: int = 8
    query: Optional[np.ndarray] = None
    walks: int = 1024
    u_ref: Optional[np.ndarray] = None
    seed: int = PHILOX_SEED
    meta: dict = dc_field(default_factory=dict)
    neumann: Optional[np.ndarray] = None     # (n_elem,) int32 flags: 1 = reflecting Neumann element
    neumann_h: Optional[np.ndarray] = None   # (n_elem,) Neumann data du/dn (n out of the domain), or None

    @property
    def dim(self) -> int:
        return int(self.vert.shape[1])

    @property
    def n_param(self) -> int:
        return 0 if self.jac is None else int(self.jac.shape[2])

    @property
    def theta0(self) -> np.ndarray:
        """Parameter vector at which `vert` is given (vertices are linear in theta)."""
        return np.asarray(self.meta.get("theta0", np.zeros(self.n_param)), dtype=np.float64)

    def reference_vertices(self) -> np.ndarray:
        """v_ref with vert = v_ref + jac @ theta0, so v(theta) = v_ref + jac theta."""
        if self.jac is None:
            return self.vert.copy()
        return self.vert - np.einsum("vkp,p->vk", self.jac, self.theta0)


def _field(c0=0.0, c=(0.0, 0.0, 0.0), A=(0.0, 0.0, 0.0, 0.0, 0.0, 0.0)) -> np.ndarray:
    return np.array([c0, *c, *A], dtype=np.float64)


# ---------------------------------------------------------------------------- 2D
def radial_polygon(n_seg: int, radius_fn, center=(0.0, 0.0)):
    t = 2 * np.pi * np.arange(n_seg) / n_seg
    r = radius_fn(t)
    vert = np.stack([center[0] + r * np.cos(t), center[1] + r * np.sin(t)], axis=1)
    elem = np.stack([np.arange(n_seg), (np.arange(n_seg) + 1) % n_seg], axis=1).astype(np.int32)
    return t, vert, elem


def fourier_jacobian(t: np.ndarray, scale: float, n_modes: int, with_radius: bool) -> np.ndarray:
    """dv/dtheta for v(t) = r(t) (cos t, sin t),
    r = [R] + scale * sum_k a_k cos kt + b_k sin kt;  theta = [R,] a_1..a_M, b_1..b_M."""
    radial = np.stack([np.cos(t), np.sin(t)], axis=1)
    cols = []
    if with_radius:
        cols.append(radial)
    for k in range(1, n_modes + 1):
        cols.append(scale * np.cos(k * t)[:, None] * radial)
    for k in range(1, n_modes + 1):
        cols.append(scale * np.sin(k * t)[:, None] * radial)
    return np.stack(cols, axis=2)


def disk_points(n: int, r_max: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    r = r_max * np.sqrt(rng.random(n))
    a = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(a), r * np.sin(a)], axis=1)


def disk_scene(variant: str = "laplace_x", n_seg: int = 128, R: float = 1.0, n_modes: int = 8,
               n_query: int = 64, walks: int = 1024, eps: float = 1e-3, h: float = 1e-2,
               K: int = 1, seed: int = GEOMETRY_SEED) -> Scene:
    """Unit-disk 128-gon, theta = [R, a_1..a_8, b_1..b_8] (all 0 at the scene).

    variant 'laplace_x': sigma = 0, restricted data g = x  (u = x, du/dtheta = 0)
    variant 'screened_1': sigma = 4, g = 1  (u = I0(2r)/I0(2R))
    variant 'mapped_cos': sigma = 0, mapped data g_v = cos t_v  (u = x/R)
    variant 'mapped_data': sigma = 0, mapped data g_v = c cos t_v + s sin t_v with
        c = 1, s = 0.5 appended to theta as boundary-data parameters:
        theta = [R, a_1..a_8, b_1..b_8, c, s], dg_v/dc = cos t_v, dg_v/ds = sin t_v
        and no vertex motion for c and s (u = (c x + s y)/R)
    """
    t, vert, elem = radial_polygon(n_seg, lambda t: np.full_like(t, R))
    jac = fourier_jacobian(t, 1.0, n_modes, with_radius=True)
    q = disk_points(n_query, 0.9 * R, seed)
    if variant == "mapped_data":
        c, s = 1.0, 0.5
        jac = np.concatenate([jac, np.zeros((n_seg, 2, 2))], axis=2)
        dg = np.zeros((n_seg, jac.shape[2]))
        dg[:, -2] = np.cos(t)
        dg[:, -1] = np.sin(t)
        sc = Scene("disk_mapped_data", vert, elem, jac, data="mapped", g_vert=c * np.cos(t) + s * np.sin(t),
                   dg_vert=dg, sigma=0.0)
        sc.eps, sc.h, sc.K, sc.query, sc.walks = eps, h, K, q, walks
        sc.meta = {"R": R, "t": t, "n_modes": n_modes, "c": c, "s": s,
                   "theta0": np.concatenate([[R], np.zeros(2 * n_modes), [c, s]])}
        return sc
    if variant == "laplace_x":
        sc = Scene("disk_laplace_x", vert, elem, jac, data="field", field=_field(c=(1.0, 0.0, 0.0)),
                   sigma=0.0)
    elif variant == "screened_1":
        sc = Scene("disk_screened_1", vert, elem, jac, data="mapped", g_vert=np.ones(n_seg), sigma=4.0)
    elif variant == "mapped_cos":
        sc = Scene("disk_mapped_cos", vert, elem, jac, data="mapped", g_vert=np.cos(t), sigma=0.0)
    else:
        raise ValueError(variant)
    sc.eps, sc.h, sc.K, sc.query, sc.walks = eps, h, K, q, walks
    sc.meta = {"R": R, "t": t, "n_modes": n_modes, "theta0": np.concatenate([[R], np.zeros(2 * n_modes)])}
    return sc


def box2d():
    vert = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]])
    elem = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], dtype=np.int32)
    return vert, elem


def box_perimeter_points(n: int, half: float) -> np.ndarray:
    """n points evenly spaced by arclength on the square |x|_inf = half."""
    side = 2 * half
    s = (np.arange(n) + 0.5) * (4 * side / n)
    pts = np.zeros((n, 2))
    for i, si in enumerate(s):
        k, r = int(si // side), si % side
        if k == 0:
            pts[i] = (-half + r, -half)
        elif k == 1:
            pts[i] = (half, -half + r)
        elif k == 2:
            pts[i] = (half - r, half)
        else:
            pts[i] = (-half, half - r)
    return pts


def star_box_scene(n_seg: int = 4096, n_modes: int = 32, coef_std: float = 0.02, base_r: float = 0.3,
                   sigma: float = 10.0, n_query: int = 256, walks: int = 4096, K: int = 2,
                   coeffs: Optional[np.ndarray] = None, seed: int = GEOMETRY_SEED) -> Scene:
    """Shape-from-diffusion in 2D: box [-1,1]^2 (g = 0) around a star emitter (g = 1).

    r(t) = base_r (1 + sum_k a_k cos kt + b_k sin kt); theta = [a_1..a_32, b_1..b_32].
    eps = 1e-3 x the bounding-cube side (2), h = 10 eps.  Observation points:
    256 points by arclength on |x|_inf = 0.9.  u_ref is the target profile of a
    round emitter of radius base_r in free space, K0(k|x|)/K0(k base_r).
    """
    rng = np.random.default_rng(seed)
    if coeffs is None:
        coeffs = rng.normal(0.0, coef_std, size=2 * n_modes)
    a, b = coeffs[:n_modes], coeffs[n_modes:]
    k = np.arange(1, n_modes + 1)

    def radius(t):
        return base_r * (1 + np.cos(np.outer(t, k)) @ a + np.sin(np.outer(t, k)) @ b)

    t, sv, se = radial_polygon(n_seg, radius)
    bv, be = box2d()
    vert = np.concatenate([bv, sv], axis=0)
    elem = np.concatenate([be, se + 4], axis=0).astype(np.int32)
    jac = np.zeros((vert.shape[0], 2, 2 * n_modes))
    jac[4:] = fourier_jacobian(t, base_r, n_modes, with_radius=False)
    g = np.concatenate([np.zeros(4), np.ones(n_seg)])
    q = box_perimeter_points(n_query, 0.9)
    from scipy.special import k0
    kap = np.sqrt(sigma)
    u_ref = k0(kap * np.linalg.norm(q, axis=1)) / k0(kap * base_r)
    eps = 1e-3 * 2.0
    sc = Scene("star_box", vert, elem, jac, data="mapped", g_vert=g, sigma=sigma, eps=eps, h=10 * eps,
               K=K, query=q, walks=walks, u_ref=u_ref)
    sc.meta = {"t": t, "coeffs": coeffs, "base_r": base_r, "theta0": np.asarray(coeffs, dtype=np.float64)}
    return sc


def translated_star_scene(offset=(0.0, 0.0), n_seg: int = 4096, n_query: int = 256, B: int = 2,
                          obs_half: float = 0.6, seed: int = GEOMETRY_SEED) -> Scene:
    """The shape-from-diffusion geometry (box [-1,1]^2 with g = 0 around the
    star emitter with g = 1, sigma = 10) with the star's position as the
    parameter: theta = the star's translation (a 2-vector, so Vector Adam
    applies), its vertices at v_ref + theta.  `offset` is the translation at
    which `vert` is given.  Observation points: n_query by arclength on the
    square |x|_inf = obs_half, near the star (the nearby slice of Sec. 5.2).
    U-statistic batches of B = 2 allow 2 walks per point."""
    sc = star_box_scene(n_seg=n_seg, n_query=n_query, seed=seed)
    sc.query = box_perimeter_points(n_query, obs_half)
    off = np.asarray(offset, dtype=np.float64)
    jac = np.zeros((sc.vert.shape[0], 2, 2))
    jac[4:, 0, 0] = 1.0
    jac[4:, 1, 1] = 1.0
    vert = sc.vert.copy()
    vert[4:] += off
    out = Scene("translated_star", vert, sc.elem, jac, data="mapped", g_vert=sc.g_vert, sigma=sc.sigma,
                eps=sc.eps, h=sc.h, K=sc.K, B=B, query=sc.query, walks=sc.walks, u_ref=sc.u_ref)
    out.meta = {"theta0": off.copy(), "coeffs": sc.meta["coeffs"]}
    return out


# ---------------------------------------------------------------------------- 3D
def icosahedron():
    p = (1 + 5 ** 0.5) / 2
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0], [0, -1, p], [0, 1, p],
                  [0, -1, -p], [0, 1, -p], [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], float)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4],
                  [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8],
                  [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosphere(freq: int):
    """Geodesic icosphere: each icosahedron face split into freq^2 triangles,
    vertices projected to the unit sphere (20 freq^2 faces, 10 freq^2 + 2 vertices)."""
    v0, f0 = icosahedron()
    ii, jj = [], []
    for i in range(freq + 1):
        for j in range(freq + 1 - i):
            ii.append(i)
            jj.append(j)
    ii, jj = np.array(ii), np.array(jj)
    index = -np.ones((freq + 1, freq + 1), dtype=np.int64)
    index[ii, jj] = np.arange(len(ii))
    tris = []
    for i in range(freq):
        for j in range(freq - i):
            tris.append((index[i, j], index[i + 1, j], index[i, j + 1]))
            if i + j < freq - 1:
                tris.append((index[i + 1, j], index[i + 1, j + 1], index[i, j + 1]))
    tris = np.array(tris, dtype=np.int64)
    A, B, C = v0[f0[:, 0]], v0[f0[:, 1]], v0[f0[:, 2]]
    pts = (A[:, None, :] + (ii / freq)[None, :, None] * (B - A)[:, None, :]
           + (jj / freq)[None, :, None] * (C - A)[:, None, :])
    pts /= np.linalg.norm(pts, axis=2, keepdims=True)
    n_local = len(ii)
    faces = (tris[None, :, :] + (np.arange(20) * n_local)[:, None, None]).reshape(-1, 3)
    flat = pts.reshape(-1, 3)
    key = np.round(flat * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    vert = flat[first]
    faces = inv.reshape(-1)[faces]
    return vert, faces.astype(np.int32)


def real_sh(lmax: int, dirs: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonics Y_lm(dirs), (n, (lmax+1)^2), order (l, m=-l..l)."""
    from scipy.special import lpmv
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    ct = np.clip(z, -1.0, 1.0)
    phi = np.arctan2(y, x)
    out = np.zeros((dirs.shape[0], (lmax + 1) ** 2))
    col = 0
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = np.sqrt((2 * l + 1) / (4 * np.pi) * factorial(l - am) / factorial(l + am))
            P = lpmv(am, l, ct)
            if m > 0:
                out[:, col] = np.sqrt(2) * norm * P * np.cos(am * phi)
            elif m < 0:
                out[:, col] = np.sqrt(2) * norm * P * np.sin(am * phi)
            else:
                out[:, col] = norm * P
            col += 1
    return out


def box3d(half: float):
    c = np.array([[x, y, z] for z in (-half, half) for y in (-half, half) for x in (-half, half)], float)
    # corners: index = x + 2y + 4z (0/1 for -/+)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, c2, d in quads:
        tris.append((a, b, c2))
        tris.append((a, c2, d))
    return c, np.array(tris, dtype=np.int32)


def sh_sphere_scene(freq: int = 100, lmax: int = 8, coef_std: float = 0.01, sigma: float = 1.0,
                    f: float = 0.5, n_query: int = 4096, walks: int = 2048, K: int = 2,
                    box_half: float = 2.0, coeffs: Optional[np.ndarray] = None,
                    eps: Optional[float] = None, seed: int = GEOMETRY_SEED) -> Scene:
    """3D thermal design: rho(w) = 1 + sum_lm c_lm Y_lm(w) on a geodesic icosphere
    (20 freq^2 triangles) inside the box [-box_half, box_half]^3.  Object g = 1,
    box g = 0, sigma = 1, constant source 0.5.  theta = c_lm (81 for lmax = 8);
    dv/dc_lm = Y_lm(w_v) w_v.  eps = 1e-3 x the bounding-cube side, h = 10 eps.
    Query points: uniform in |x|_inf < box_half - 0.1, outside the analytic
    surface by at least 0.02."""
    rng = np.random.default_rng(seed)
    nsh = (lmax + 1) ** 2
    if coeffs is None:
        coeffs = rng.normal(0.0, coef_std, size=nsh)
    dirs, faces = icosphere(freq)
    Y = real_sh(lmax, dirs)
    rho = 1.0 + Y @ coeffs
    sv = dirs * rho[:, None]
    bv, be = box3d(box_half)
    nb = bv.shape[0]
    vert = np.concatenate([bv, sv], axis=0)
    elem = np.concatenate([be, faces + nb], axis=0).astype(np.int32)
    jac = np.zeros((vert.shape[0], 3, nsh))
    jac[nb:] = Y[:, None, :] * dirs[:, :, None]
    g = np.concatenate([np.zeros(nb), np.ones(sv.shape[0])])
    lim = box_half - 0.1
    pts = []
    while sum(len(p) for p in pts) < n_query:
        c = rng.uniform(-lim, lim, size=(4 * n_query, 3))
        r = np.linalg.norm(c, axis=1)
        d = c / np.maximum(r, 1e-12)[:, None]
        rr = 1.0 + real_sh(lmax, d) @ coeffs
        pts.append(c[r > rr + 0.02])
    q = np.concatenate(pts, axis=0)[:n_query]
    if eps is None:
        eps = 1e-3 * 2 * box_half
    sc = Scene("sh_sphere_box", vert, elem, jac, data="mapped", g_vert=g, sigma=sigma, f=f, eps=eps,
               h=10 * eps, K=K, query=q, walks=walks)
    sc.meta = {"coeffs": coeffs, "lmax": lmax, "freq": freq, "dirs": dirs,
               "theta0": np.asarray(coeffs, dtype=np.float64)}
    return sc


def ball_scene(freq: int = 16, R: float = 1.0, sigma: float = 1.0, f: float = 0.0, g: float = 1.0,
               n_query: int = 16, walks: int = 256, eps: float = 1e-3, h: float = 1e-2, K: int = 1,
               seed: int = GEOMETRY_SEED) -> Scene:
    """Icosphere of radius R (theta = [R], dv/dR = w_v) with constant data g."""
    dirs, faces = icosphere(freq)
    vert = R * dirs
    jac = dirs[:, :, None].copy()
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_query, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 0.8 * R * rng.random(n_query) ** (1 / 3)
    q = d * r[:, None]
    sc = Scene("ball", vert, faces, jac, data="mapped", g_vert=np.full(vert.shape[0], g), sigma=sigma,
               f=f, eps=eps, h=h, K=K, query=q, walks=walks)
    sc.meta = {"R": R, "theta0": np.array([R])}
    return sc


def batched_problems(n: int = 64, seed: int = GEOMETRY_SEED, scale: float = 1.0, max_elems: int = 500_000):
    """Batched workload: n independent problems, half 2D star-in-box, half 3D
    SH-sphere-in-box, with element counts log-uniform in [1e3, max_elems],
    query counts log-uniform in [16, 4096] (times `scale`), sigma log-uniform in
    [0.01, 100], walks per point 2^floor(U[8, 12]) (times `scale`, kept a
    multiple of 8), and 16 shape parameters (Fourier k <= 8 in 2D, SH l <= 3 in
    3D).  Each scene carries query points, walks and a target u_ref."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_el = int(np.exp(rng.uniform(np.log(1e3), np.log(max_elems))))
        n_q = max(16, int(np.exp(rng.uniform(np.log(16), np.log(4096))) * scale))
        sigma = float(np.exp(rng.uniform(np.log(0.01), np.log(100.0))))
        walks = max(8, int(2 ** int(rng.uniform(8, 12.999)) * scale) // 8 * 8)
        sub = int(rng.integers(0, 2 ** 31))
        if i % 2 == 0:
            sc = star_box_scene(n_seg=max(64, n_el - 4), n_modes=8, sigma=sigma, n_query=n_q, walks=walks, seed=sub)
        else:
            freq = max(7, int(round(np.sqrt(max(n_el - 12, 20) / 20.0))))
            sc = sh_sphere_scene(freq=freq, lmax=3, coef_std=0.02, sigma=sigma, n_query=n_q, walks=walks, seed=sub)
            sc.u_ref = np.zeros(n_q)
        sc.name = f"batch{i:02d}_{sc.dim}d"
        out.append(sc)
    return out


# ------------------------------------------------------------- mixed boundaries
def _polyline(points):
    """Vertices of consecutive point lists joined end to start (a closed loop)."""
    v = np.concatenate(points, axis=0)
    n = v.shape[0]
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    return v, e


def quarter_disk_scene(data: str = "field", n_arc: int = 128, n_axis: int = 16, n_query: int = 12,
                       walks: int = 1024, eps: float = 1e-3, h: float = 1e-2, K: int = 1,
                       seed: int = GEOMETRY_SEED) -> Scene:
    """Quarter disk {r < R, 0 < angle < pi/2}, R = 1: the arc (n_arc segments) is
    Dirichlet, the two radii on the axes (n_axis segments each) reflecting
    Neumann.  theta = [R] scales every vertex (the arc moves along its normal,
    the radii along themselves).  data 'field': g = x^2 - y^2 (restricted);
    'mapped': g_v = cos 2 t_v on the arc."""
    t = 0.5 * np.pi * np.arange(n_arc + 1) / n_arc
    arc = np.stack([np.cos(t), np.sin(t)], 1)                       # (1, 0) .. (0, 1)
    yv = 1.0 - np.arange(1, n_axis + 1) / n_axis                    # (0, y) down to the origin
    xv = np.arange(1, n_axis) / n_axis                              # (x, 0) up to (1, 0), excluded
    vert, elem = _polyline([arc, np.stack([0 * yv, yv], 1), np.stack([xv, 0 * xv], 1)])
    neumann = np.zeros(len(elem), np.int32)
    neumann[n_arc:] = 1
    jac = vert[:, :, None].copy()
    ang = np.arctan2(vert[:, 1], vert[:, 0])
    rng = np.random.default_rng(seed)
    r = 0.15 + 0.7 * rng.random(n_query)
    a = 0.1 + (0.5 * np.pi - 0.2) * rng.random(n_query)
    q = np.stack([r * np.cos(a), r * np.sin(a)], 1)
    if data == "field":
        sc = Scene("quarter_disk_field", vert, elem, jac, data="field",
                   field=_field(A=(1.0, -1.0, 0.0, 0.0, 0.0, 0.0)), sigma=0.0)
    else:
        sc = Scene("quarter_disk_mapped", vert, elem, jac, data="mapped", g_vert=np.cos(2 * ang), sigma=0.0)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, neumann
    sc.meta = {"theta0": np.array([1.0])}
    return sc


def strip_scene(sigma: float = 4.0, f: float = 0.0, g: float = 1.0, half: float = 0.5, n_side: int = 16,
                n_tb: int = 32, n_query: int = 12, walks: int = 1024, eps: float = 1e-3, h: float = 1e-2,
                K: int = 1, seed: int = GEOMETRY_SEED) -> Scene:
    """Rectangle [-1, 1] x [-half, half]: the sides x = -1 and x = L (L = 1) are
    Dirichlet with mapped data g, the bottom and top reflecting Neumann.
    theta = [L] moves the right side (its vertices, the corners included, move
    in x; the top and bottom stretch along themselves)."""
    bx = -1.0 + 2.0 * np.arange(n_tb) / n_tb
    ry = -half + 2 * half * np.arange(n_side) / n_side
    vert, elem = _polyline([np.stack([bx, np.full(n_tb, -half)], 1), np.stack([np.ones(n_side), ry], 1),
                            np.stack([-bx, np.full(n_tb, half)], 1), np.stack([-np.ones(n_side), -ry], 1)])
    neumann = np.zeros(len(elem), np.int32)
    neumann[:n_tb] = 1
    neumann[n_tb + n_side:2 * n_tb + n_side] = 1
    jac = np.zeros((len(vert), 2, 1))
    jac[np.isclose(vert[:, 0], 1.0), 0, 0] = 1.0
    rng = np.random.default_rng(seed)
    q = np.stack([rng.uniform(-0.9, 0.9, n_query), rng.uniform(-0.8 * half, 0.8 * half, n_query)], 1)
    sc = Scene("strip", vert, elem, jac, data="mapped", g_vert=np.full(len(vert), g), sigma=sigma, f=f)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, neumann
    sc.meta = {"theta0": np.array([1.0]), "g": g}
    return sc


def slit_disk_scene(n_circle: int = 256, n_slit: int = 32, n_query: int = 12, walks: int = 1024,
                    eps: float = 1e-3, seed: int = GEOMETRY_SEED) -> Scene:
    """Unit disk cut along the slit [0, 1) x {0}: the circle is Dirichlet with
    mapped data g(t) = cos(t / 2), t in [0, 2 pi] (the vertex at (1, 0) is
    doubled so that the data can jump there), the slit is a reflecting
    Neumann boundary seen from both sides, open at the origin.  No shape
    parameters."""
    t = 2 * np.pi * np.arange(n_circle + 1) / n_circle
    circ = np.stack([np.cos(t), np.sin(t)], 1)
    sv = np.stack([np.arange(n_slit + 1) / n_slit, np.zeros(n_slit + 1)], 1)
    vert = np.concatenate([circ, sv], 0)
    ce = np.stack([np.arange(n_circle), np.arange(1, n_circle + 1)], 1)
    se = n_circle + 1 + np.stack([np.arange(n_slit), np.arange(1, n_slit + 1)], 1)
    elem = np.concatenate([ce, se], 0).astype(np.int32)
    neumann = np.concatenate([np.zeros(n_circle), np.ones(n_slit)]).astype(np.int32)
    g = np.concatenate([np.cos(t / 2), np.zeros(n_slit + 1)])
    rng = np.random.default_rng(seed)
    r = 0.25 + 0.55 * rng.random(n_query)
    a = 0.3 + (2 * np.pi - 0.6) * rng.random(n_query)
    q = np.stack([r * np.cos(a), r * np.sin(a)], 1)
    sc = Scene("slit_disk", vert, elem, None, data="mapped", g_vert=g, sigma=0.0)
    sc.eps, sc.query, sc.walks, sc.neumann = eps, q, walks, neumann
    return sc


def thermal_scene(offset=(0.0, 0.0), n_wire: int = 64, n_slab: int = 40, n_query: int = 32, walks: int = 1024,
                  eps: float = 1e-3, h: float = 1e-2, K: int = 2, seed: int = GEOMETRY_SEED) -> Scene:
    """A 2D thermal design in the manner of Sec. 6.3: a heating wire (a circle of
    radius 0.06 around (0, -0.35), n_wire segments, Dirichlet g = 1) warms an
    insulating slab ([-0.5, 0.5] x [0.2, 0.3], a closed polyline of n_slab
    segments per long side, reflecting Neumann) inside the box [-1, 1]^2 held
    at g = 0; sigma = 0, no source.  theta = the wire's translation (a
    2-vector: Vector Adam applies), at `offset` in `vert`.  Observation points:
    n_query points on the slab's underside y = 0.2 (on the Neumann part, where
    the thermal design reads its temperatures)."""
    bv, be = box2d()
    t = 2 * np.pi * np.arange(n_wire) / n_wire
    wire = np.stack([0.06 * np.cos(t), -0.35 + 0.06 * np.sin(t)], 1) + np.asarray(offset, dtype=np.float64)
    xs = -0.5 + np.arange(n_slab) / n_slab
    n_end = 4
    ye = 0.2 + 0.1 * np.arange(n_end) / n_end
    slab = np.concatenate([np.stack([xs, np.full(n_slab, 0.2)], 1), np.stack([np.full(n_end, 0.5), ye], 1),
                           np.stack([-xs, np.full(n_slab, 0.3)], 1), np.stack([np.full(n_end, -0.5), 0.5 - ye], 1)])
    ws = np.stack([np.arange(n_wire), (np.arange(n_wire) + 1) % n_wire], 1) + 4
    ns = len(slab)
    ss = np.stack([np.arange(ns), (np.arange(ns) + 1) % ns], 1) + 4 + n_wire
    vert = np.concatenate([bv, wire, slab], 0)
    elem = np.concatenate([be, ws, ss], 0).astype(np.int32)
    neumann = np.concatenate([np.zeros(4 + n_wire), np.ones(ns)]).astype(np.int32)
    g = np.concatenate([np.zeros(4), np.ones(n_wire), np.zeros(ns)])
    jac = np.zeros((len(vert), 2, 2))
    jac[4:4 + n_wire, 0, 0] = 1.0
    jac[4:4 + n_wire, 1, 1] = 1.0
    qx = -0.45 + 0.9 * (np.arange(n_query) + 0.5) / n_query
    q = np.stack([qx, np.full(n_query, 0.2)], 1)
    sc = Scene("thermal", vert, elem, jac, data="mapped", g_vert=g, sigma=0.0)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, neumann
    sc.meta = {"theta0": np.asarray(offset, dtype=np.float64)}
    return sc


def cylinder_flow_scene(a: float = 0.4, n_circle: int = 300, n_side: int = 64, n_query: int = 8,
                        walks: int = 1024, eps: float = 1e-3, h: float = 1e-2, K: int = 1,
                        seed: int = GEOMETRY_SEED) -> Scene:
    """Potential flow past a cylinder: the box [-1, 1]^2 (n_side segments per
    side, Dirichlet, mapped data g = x (1 + a^2 / r^2) at the vertices, scaled
    by one data parameter c at c = 1) around an insulating circle of radius a
    (n_circle segments, reflecting Neumann; every vertex a silhouette
    candidate).  u = x (1 + a^2 / r^2) in the domain, du/dc = u.  Query points
    uniform in |x|_inf < 0.9 with r > a + 0.05."""
    t = np.linspace(-1.0, 1.0, n_side + 1)[:-1]
    box = np.concatenate([np.stack([t, np.full(n_side, -1.0)], 1), np.stack([np.full(n_side, 1.0), t], 1),
                          np.stack([-t, np.full(n_side, 1.0)], 1), np.stack([np.full(n_side, -1.0), -t], 1)])
    nb = len(box)
    ph = 2 * np.pi * np.arange(n_circle) / n_circle
    circ = a * np.stack([np.cos(ph), np.sin(ph)], 1)
    vert = np.concatenate([box, circ], 0)
    elem = np.concatenate([np.stack([np.arange(nb), (np.arange(nb) + 1) % nb], 1),
                           np.stack([np.arange(n_circle), (np.arange(n_circle) + 1) % n_circle], 1) + nb]).astype(np.int32)
    neumann = np.concatenate([np.zeros(nb), np.ones(n_circle)]).astype(np.int32)
    g = vert[:, 0] * (1.0 + a * a / (vert[:, 0] ** 2 + vert[:, 1] ** 2))
    rng = np.random.default_rng(seed)
    q = np.zeros((0, 2))
    while len(q) < n_query:
        p = rng.uniform(-0.9, 0.9, size=(4 * n_query, 2))
        q = np.concatenate([q, p[np.hypot(p[:, 0], p[:, 1]) > a + 0.05]])[:n_query]
    sc = Scene("cylinder_flow", vert, elem, np.zeros((len(vert), 2, 1)), data="mapped", g_vert=g,
               dg_vert=g[:, None].copy(), sigma=0.0)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, neumann
    sc.meta = {"a": a}
    return sc


def neumann_data_box_scene(dim: int = 2, c: float = 0.5, b: float = 0.3, n_side: int = 16, m: int = 4,
                           n_query: int = 8, walks: int = 1024, eps: float = 1e-3, h: float = 1e-2, K: int = 1,
                           seed: int = GEOMETRY_SEED) -> Scene:
    """Neumann data on the box [-1, 1]^dim: the faces x = -1 and x = X (X = 1)
    Dirichlet with the restricted data g = b x + c (y^2 - x^2) (2D) or
    b x + c (y^2 + z^2 - 2 x^2) (3D), the other faces Neumann with data
    du/dn = 2c (n out of the box); u = g.  2D: n_side segments per side; 3D:
    2 m^2 triangles per face.  theta = [X] moves the face x = X."""
    if dim == 2:
        sc = strip_scene(sigma=0.0, half=1.0, n_side=n_side, n_tb=n_side, n_query=n_query, walks=walks, eps=eps,
                         h=h, K=K, seed=seed)
        sc.field = _field(c=(b, 0.0, 0.0), A=(-c, c, 0.0, 0.0, 0.0, 0.0))
    else:
        sc = cube_neumann_scene(m=m, n_query=n_query, walks=walks, eps=eps, h=h, K=K, seed=seed)
        sc.field = _field(c=(b, 0.0, 0.0), A=(-2 * c, c, c, 0.0, 0.0, 0.0))
    sc.name = "neumann_data_box_%dd" % dim
    sc.data, sc.g_vert = "field", None
    sc.neumann_h = np.where(sc.neumann == 1, 2.0 * c, 0.0)
    sc.meta.update(c=c, b=b)
    return sc


def screened_neumann_data_box_scene(k: float = 1.5, s: float = 0.5, n_side: int = 32, n_query: int = 8,
                                    walks: int = 1024, eps: float = 1e-3, h: float = 1e-2, K: int = 1,
                                    seed: int = GEOMETRY_SEED) -> Scene:
    """The square [-1, 1]^2 with -Lap u + k^2 u = 0: the sides x = -1 and
    x = X (X = 1) Dirichlet with mapped data cosh(k y) -/+ s sinh(k) at their
    vertices, the sides y = -1, 1 Neumann with data du/dn = k sinh(k);
    u = cosh(k y) + s sinh(k x).  theta = [X] moves the side x = X."""
    sc = strip_scene(sigma=k * k, half=1.0, n_side=n_side, n_tb=n_side, n_query=n_query, walks=walks, eps=eps,
                     h=h, K=K, seed=seed)
    sc.name = "screened_neumann_data_box"
    v = sc.vert
    sc.g_vert = np.cosh(k * v[:, 1]) + s * np.sinh(k) * np.sign(v[:, 0])
    sc.neumann_h = np.where(sc.neumann == 1, k * np.sinh(k), 0.0)
    sc.meta.update(k=k, s=s)
    return sc


def annulus_neumann_data_scene(r_in: float = 0.4, n_in: int = 128, n_out: int = 128, a: float = 1.0,
                               b: float = 0.5, n_query: int = 8, walks: int = 1024, eps: float = 1e-3,
                               seed: int = GEOMETRY_SEED) -> Scene:
    """The annulus r_in < r < 1: the outer circle (n_out segments) Dirichlet
    with mapped data a, the inner circle (n_in segments) Neumann with data
    du/dn = -b / r_in (n out of the domain, towards the centre); u = a + b log r.
    No shape parameters.  Query points with r in (r_in + 0.05, 0.9)."""
    t1 = 2 * np.pi * np.arange(n_out) / n_out
    t2 = 2 * np.pi * np.arange(n_in) / n_in
    vert = np.concatenate([np.stack([np.cos(t1), np.sin(t1)], 1), r_in * np.stack([np.cos(t2), np.sin(t2)], 1)])
    elem = np.concatenate([np.stack([np.arange(n_out), (np.arange(n_out) + 1) % n_out], 1),
                           n_out + np.stack([np.arange(n_in), (np.arange(n_in) + 1) % n_in], 1)]).astype(np.int32)
    neumann = np.concatenate([np.zeros(n_out), np.ones(n_in)]).astype(np.int32)
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_in + 0.05, 0.9, n_query)
    ph = rng.uniform(0.0, 2 * np.pi, n_query)
    sc = Scene("annulus_neumann_data", vert, elem, None, data="mapped", g_vert=np.full(len(vert), a), sigma=0.0)
    sc.eps, sc.query, sc.walks, sc.neumann = eps, np.stack([r * np.cos(ph), r * np.sin(ph)], 1), walks, neumann
    sc.neumann_h = np.where(neumann == 1, -b / r_in, 0.0)
    sc.meta = {"a": a, "b": b, "r_in": r_in}
    return sc


def box3d_grid(m: int, half: float = 1.0):
    """The cube [-half, half]^3 with each face split into 2 m^2 triangles
    (shared vertices merged)."""
    pts, tris = [], []
    u = np.linspace(-half, half, m + 1)
    for axis in range(3):
        for sgn in (-half, half):
            a, b = [k for k in range(3) if k != axis]
            base = sum(len(p) for p in pts)
            P = np.zeros(((m + 1) ** 2, 3))
            P[:, axis] = sgn
            P[:, a] = np.repeat(u, m + 1)
            P[:, b] = np.tile(u, m + 1)
            pts.append(P)
            for i in range(m):
                for j in range(m):
                    p0 = base + i * (m + 1) + j
                    tris += [(p0, p0 + m + 1, p0 + 1), (p0 + 1, p0 + m + 1, p0 + m + 2)]
    flat = np.concatenate(pts, 0)
    key = np.round(flat * 1e6).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    return flat[first], inv.reshape(-1)[np.array(tris)].astype(np.int32)


def box_grid(lo, hi, m: int):
    """The box [lo, hi] (3-vectors) with each face split into 2 m^2 triangles,
    wound consistently (normals out of the box; shared vertices merged)."""
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    v, e = box3d_grid(m, 1.0)
    vert = lo + 0.5 * (v + 1.0) * (hi - lo)
    # orient every triangle's normal away from the box centre
    c = 0.5 * (lo + hi)
    a, b, cc = vert[e[:, 0]], vert[e[:, 1]], vert[e[:, 2]]
    n = np.cross(b - a, cc - a)
    flip = np.sum(n * ((a + b + cc) / 3.0 - c), axis=1) < 0
    e = e.copy()
    e[flip] = e[flip][:, [0, 2, 1]]
    return vert, e


def thermal_scene_3d(offset=(0.0, 0.0, 0.0), freq: int = 4, slab_m: int = 4, box_m: int = 2, n_side: int = 6,
                     walks: int = 1024, eps: float = 1e-3, h: float = 1e-2, K: int = 2,
                     seed: int = GEOMETRY_SEED) -> Scene:
    """The thermal design of Sec. 6.3 in 3D: a heating element (a sphere of
    radius 0.1 around (0, 0, -0.35), an icosphere of 20 freq^2 triangles,
    Dirichlet g = 1) warms an insulating slab ([-0.5, 0.5]^2 x [0.2, 0.3], its
    faces split into 2 slab_m^2 triangles each, reflecting Neumann) inside the
    box [-1, 1]^3 held at g = 0; sigma = 0, no source.  theta = the heater's
    translation (a 3-vector: Vector Adam applies), at `offset` in `vert`.
    Observation points: an n_side x n_side grid on the slab's underside z = 0.2
    (on the Neumann part)."""
    bv, be = box3d_grid(box_m)
    hv, he = icosphere(freq)
    hv = 0.1 * hv + np.array([0.0, 0.0, -0.35]) + np.asarray(offset, dtype=np.float64)
    sv, se = box_grid((-0.5, -0.5, 0.2), (0.5, 0.5, 0.3), slab_m)
    vert = np.concatenate([bv, hv, sv], 0)
    nb, nh = len(bv), len(hv)
    elem = np.concatenate([be, he + nb, se + nb + nh]).astype(np.int32)
    neumann = np.concatenate([np.zeros(len(be) + len(he)), np.ones(len(se))]).astype(np.int32)
    g = np.concatenate([np.zeros(nb), np.ones(nh), np.zeros(len(sv))])
    jac = np.zeros((len(vert), 3, 3))
    for k in range(3):
        jac[nb:nb + nh, k, k] = 1.0
    t = -0.4 + 0.8 * (np.arange(n_side) + 0.5) / n_side
    q = np.stack([np.repeat(t, n_side), np.tile(t, n_side), np.full(n_side * n_side, 0.2)], 1)
    sc = Scene("thermal_3d", vert, elem, jac, data="mapped", g_vert=g, sigma=0.0)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, neumann
    sc.meta = {"theta0": np.asarray(offset, dtype=np.float64)}
    return sc


def sphere_flow_scene(a: float = 0.4, freq: int = 6, m: int = 8, n_query: int = 8, walks: int = 1024,
                      eps: float = 1e-3, h: float = 1e-2, K: int = 1, r_min: float = 0.6, q: float = 0.0,
                      seed: int = GEOMETRY_SEED) -> Scene:
    """Potential flow past a sphere in 3D: the box [-1, 1]^3 (2 m^2 triangles
    per face, Dirichlet, mapped data g = x (1 + a^3 / (2 r^3)) at the vertices,
    scaled by one data parameter c at c = 1) around an insulating geodesic
    icosphere of radius a (20 freq^2 triangles, reflecting Neumann; every edge
    a silhouette candidate).  u = x (1 + a^3 / (2 r^3)) in the domain,
    du/dc = u.  With q != 0 the sphere also emits a point-source flow: Neumann
    data du/dn = q / a^2 on it (n out of the domain, towards the centre) and
    q / r added to the box's data, not scaled by c; u gains q / r, du/dc stays
    the flow.  Query points uniform in |x|_inf < 0.9 with r > r_min."""
    bv, be = box3d_grid(m)
    sv, se = icosphere(freq)
    vert = np.concatenate([bv, a * sv], 0)
    elem = np.concatenate([be, se + len(bv)]).astype(np.int32)
    neumann = np.concatenate([np.zeros(len(be)), np.ones(len(se))]).astype(np.int32)
    r3 = np.sum(vert * vert, axis=1) ** 1.5
    g = vert[:, 0] * (1.0 + a ** 3 / (2.0 * r3))
    rng = np.random.default_rng(seed)
    pts = np.zeros((0, 3))
    while len(pts) < n_query:
        p = rng.uniform(-0.9, 0.9, size=(4 * n_query, 3))
        pts = np.concatenate([pts, p[np.linalg.norm(p, axis=1) > r_min]])[:n_query]
    g_all = g + (q / np.cbrt(r3) if q else 0.0)
    sc = Scene("sphere_flow", vert, elem, np.zeros((len(vert), 3, 1)), data="mapped", g_vert=g_all,
               dg_vert=g[:, None].copy(), sigma=0.0)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, pts, walks, neumann
    if q:
        sc.neumann_h = np.where(neumann == 1, q / (a * a), 0.0)
    sc.meta = {"a": a, "q": q}
    return sc


def cube_neumann_scene(m: int = 4, n_query: int = 8, walks: int = 1024, eps: float = 1e-3, h: float = 1e-2,
                       K: int = 1, sigma: float = 0.0, f: float = 0.0, seed: int = GEOMETRY_SEED) -> Scene:
    """Cube [-1, 1]^3, each face split into 2 m^2 triangles: the faces x = -1 and
    x = X (X = 1) are Dirichlet with mapped data g = x (-1 and 1), the other
    four reflecting Neumann; constant source f of -Lap u + sigma u = f.
    theta = [X] moves the face x = X (its vertices move in x; the side faces
    stretch along themselves)."""
    pts, tris, flags = [], [], []
    u = np.linspace(-1.0, 1.0, m + 1)
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            a, b = [k for k in range(3) if k != axis]
            base = sum(len(p) for p in pts)
            P = np.zeros(((m + 1) ** 2, 3))
            P[:, axis] = sgn
            P[:, a] = np.repeat(u, m + 1)
            P[:, b] = np.tile(u, m + 1)
            pts.append(P)
            for i in range(m):
                for j in range(m):
                    p0 = base + i * (m + 1) + j
                    tris += [(p0, p0 + m + 1, p0 + 1), (p0 + 1, p0 + m + 1, p0 + m + 2)]
                    flags += [0 if axis == 0 else 1] * 2
    flat = np.concatenate(pts, 0)
    key = np.round(flat * 1e6).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    vert = flat[first]
    elem = inv.reshape(-1)[np.array(tris)].astype(np.int32)
    jac = np.zeros((len(vert), 3, 1))
    jac[np.isclose(vert[:, 0], 1.0), 0, 0] = 1.0
    rng = np.random.default_rng(seed)
    q = rng.uniform(-0.8, 0.8, size=(n_query, 3))
    sc = Scene("cube_neumann", vert, elem, jac, data="mapped", g_vert=vert[:, 0].copy(), sigma=sigma, f=f)
    sc.eps, sc.h, sc.K, sc.query, sc.walks, sc.neumann = eps, h, K, q, walks, np.array(flags, np.int32)
    sc.meta = {"theta0": np.array([1.0])}
    return sc
