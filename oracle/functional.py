"""FP64 reference of the volume-integrated shape functional (test
infrastructure only).

J(theta) = int_Omega M(x) 1/2 (u(x) - uref(x))^2 dx          (Eq. functional)
dJ/dtheta = int_Omega M (u - uref) udot dx
          + int_Gamma M V_n 1/2 (u - uref)^2 dA              (Eq. functional_deriv)

with M the indicator of an axis-aligned box.  The domain integral is the
Monte Carlo estimate over n_try points uniform in the box, those inside Omega
weighted |box| / n_try each; the boundary integral has u = g (Dirichlet data)
and is integrated exactly per element from the barycentric monomial integrals
  segment:  int w0^i w1^j ds    = L i! j! / (i + j + 1)!
  triangle: int w0^i w1^j w2^k dA = 2 A i! j! k! / (i + j + k + 2)!
Readings shared with the library: M on the boundary is the box indicator at
the element's centre; the outward normal is the element's normal oriented so
that the point 1e-3 of the element's size behind its centre is inside; the
domain points come from Philox4x32-10 with key = seed and counter
(i, 0, 0, 0xD0A1), words 0..dim-1 mapped to (0, 1) as for the walks.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import Problem, inside, philox4x32_10, uniform
from . import estimators as est


def sample_domain(prob: Problem, n_try: int, box_lo, box_hi, seed: int):
    """Candidates uniform in the box, kept (in order) if inside Omega; returns
    (points, weight per point)."""
    lo = np.asarray(box_lo, dtype=np.float64)[:prob.dim]
    hi = np.asarray(box_hi, dtype=np.float64)[:prob.dim]
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    cand = np.empty((n_try, prob.dim))
    for i in range(n_try):
        w = philox4x32_10(np.array([i, 0, 0, 0xD0A1], dtype=np.uint32), key)
        for k in range(prob.dim):
            cand[i, k] = lo[k] + (hi[k] - lo[k]) * uniform(int(w[k]))
    keep = inside(prob, cand)
    return cand[keep], float(np.prod(hi - lo) / n_try)


def grad_l2_weighted(u_hat, udot, u_ref, weights, n_points: int, W: int, B: int) -> np.ndarray:
    """sum_p w_p times the U-statistic gradient of 1/2 (u_p - uref_p)^2 (Eq. ustatistics)."""
    g = np.zeros(np.shape(udot)[1])
    u = np.asarray(u_hat).reshape(n_points, W)
    ud = np.asarray(udot).reshape(n_points, W, -1)
    for p in range(n_points):
        g += weights[p] * est.grad_l2_ustat(u[p], ud[p], [u_ref[p]], 1, W, B)
    return g


def loss_l2_weighted(u_hat, u_ref, weights, n_points: int, W: int) -> float:
    m = np.asarray(u_hat).reshape(n_points, W).mean(axis=1)
    return float(np.sum(np.asarray(weights) * 0.5 * (m - np.asarray(u_ref)) ** 2))


def _simplex_monomial(measure: float, exps) -> float:
    """Integral of prod_a w_a^exps[a] over a segment (2 exponents, measure =
    length) or a triangle (3 exponents, measure = area)."""
    n = len(exps)
    num = np.prod([factorial(e) for e in exps])
    return measure * factorial(n - 1) * num / factorial(sum(exps) + n - 1)


def boundary_term_l2(prob: Problem, box_lo, box_hi, uref_vert=None) -> np.ndarray:
    """int_Gamma M V_n 1/2 (g - uref)^2 dA per parameter, for mapped vertex data."""
    dim = prob.dim
    vert = np.asarray(prob.vert, dtype=np.float64).reshape(-1, dim)
    elem = np.asarray(prob.elem).reshape(-1, dim)
    g = np.asarray(prob.g_vert, dtype=np.float64)
    ur = np.zeros(len(vert)) if uref_vert is None else np.asarray(uref_vert, dtype=np.float64)
    lo = np.asarray(box_lo, dtype=np.float64)[:dim]
    hi = np.asarray(box_hi, dtype=np.float64)[:dim]
    jac = np.asarray(prob.jac, dtype=np.float64).reshape(len(vert), dim, -1)
    # outward orientation: the point just behind the centre is inside
    normals, sizes, centres = [], [], []
    for e in elem:
        v = vert[e]
        c = v.mean(axis=0)
        if dim == 2:
            t = v[1] - v[0]
            n = np.array([t[1], -t[0]])
            size, measure = np.linalg.norm(t), np.linalg.norm(t)
        else:
            n = np.cross(v[1] - v[0], v[2] - v[0])
            size, measure = np.sqrt(np.linalg.norm(n)), 0.5 * np.linalg.norm(n)
        normals.append(n / np.linalg.norm(n))
        sizes.append((size, measure))
        centres.append(c)
    normals = np.array(normals)
    centres = np.array(centres)
    behind = centres - 1e-3 * np.array([s for s, _ in sizes])[:, None] * normals
    sgn = np.where(inside(prob, behind), 1.0, -1.0)
    acc = np.zeros((len(vert), dim))
    for ei, e in enumerate(elem):
        c = centres[ei]
        if not (np.all(c >= lo) and np.all(c <= hi)):
            continue
        measure = sizes[ei][1]
        d = g[e] - ur[e]
        for a in range(dim):
            # int w_a 1/2 (sum_b w_b d_b)^2 = 1/2 sum_{b,c} d_b d_c int w_a w_b w_c
            total = 0.0
            for b in range(dim):
                for cc in range(dim):
                    exps = [0] * dim
                    exps[a] += 1
                    exps[b] += 1
                    exps[cc] += 1
                    total += 0.5 * d[b] * d[cc] * _simplex_monomial(measure, exps)
            acc[e[a]] += sgn[ei] * total * normals[ei]
    return np.einsum("vk,vkp->p", acc, jac)


# ---------------------------------------------------------------------------
# Boundary loss of the general shape functional (App. C, Eq. general_functional):
#   J_b(theta) = int_Gamma m(y) l_b(u(y)) dA(y),   l_b(u) = 1/2 (u - ub_ref)^2.
# Its derivative (Eq. general_functional_deriv) has, on Gamma, the terms
#   m [ udot l_b'(u) + V_n (kappa l_b(u) + l_b'(u) du/dn) ].
# On a Dirichlet boundary u = g and, by the boundary condition of the
# differential BVP (Eq. bvp_deriv), udot = gdot - V_n du/dn (with dg/dn = 0 for
# mapped data), so the du/dn terms cancel and no walk is needed: what remains
# is the derivative of int_Gamma m l_b(g) dA along the boundary motion and the
# data derivative.  For a boundary of segments or triangles with g and ub_ref
# linear on each element, the mean-curvature term kappa V_n l_b is the
# derivative of the element measures, so the functional is differentiated
# exactly as the sum over elements of m_e |e| Q_e, where |e| is the element's
# length or area and Q_e = int over the reference element of l_b (the mean of
# l_b over e).  m_e is the box indicator at the element's centre and is held
# fixed (the masks are fixed functions in App. C).
def _measure_and_gradient(v: np.ndarray):
    """Length or area of an element with vertices v (2 x 2 or 3 x 3) and its
    gradient with respect to each vertex (same shape as v)."""
    if v.shape[0] == 2:
        t = v[1] - v[0]
        L = np.linalg.norm(t)
        return L, np.stack([-t / L, t / L])
    a, b, c = v
    n = np.cross(b - a, c - a)
    nn = np.linalg.norm(n)
    nh = n / nn
    # dA/da = 1/2 nhat x (c - b), cyclically
    return 0.5 * nn, 0.5 * np.stack([np.cross(nh, c - b), np.cross(nh, a - c), np.cross(nh, b - a)])


def _mean_half_square(d: np.ndarray) -> float:
    """Mean over a segment / triangle of 1/2 (sum_a w_a d_a)^2 (barycentrics w)."""
    n = len(d)
    tot = 0.0
    for a in range(n):
        for b in range(n):
            exps = [0] * n
            exps[a] += 1
            exps[b] += 1
            tot += 0.5 * d[a] * d[b] * _simplex_monomial(1.0, exps)
    return tot


def _element_masked(prob: Problem, box_lo, box_hi):
    dim = prob.dim
    vert = np.asarray(prob.vert, dtype=np.float64).reshape(-1, dim)
    elem = np.asarray(prob.elem).reshape(-1, dim)
    lo = np.asarray(box_lo, dtype=np.float64)[:dim]
    hi = np.asarray(box_hi, dtype=np.float64)[:dim]
    c = vert[elem].mean(axis=1)
    return vert, elem, np.all((c >= lo) & (c <= hi), axis=1)


def boundary_loss_l2_value(prob: Problem, box_lo, box_hi, ub_vert=None) -> float:
    """J_b = sum_e m_e int_e 1/2 (g - ub)^2 dA, integrated exactly per element."""
    vert, elem, m = _element_masked(prob, box_lo, box_hi)
    g = np.asarray(prob.g_vert, dtype=np.float64)
    ub = np.zeros(len(vert)) if ub_vert is None else np.asarray(ub_vert, dtype=np.float64)
    tot = 0.0
    for ei, e in enumerate(elem):
        if not m[ei]:
            continue
        meas, _ = _measure_and_gradient(vert[e])
        tot += meas * _mean_half_square(g[e] - ub[e])
    return float(tot)


def boundary_loss_l2(prob: Problem, box_lo, box_hi, ub_vert=None):
    """(J_b, dJ_b/dtheta) for mapped vertex data g (derivative dg_vert, or
    none) and vertices moving with the Jacobian jac (n_vert x dim x N)."""
    vert, elem, m = _element_masked(prob, box_lo, box_hi)
    dim = prob.dim
    g = np.asarray(prob.g_vert, dtype=np.float64)
    ub = np.zeros(len(vert)) if ub_vert is None else np.asarray(ub_vert, dtype=np.float64)
    N = prob.n_param
    jac = np.zeros((len(vert), dim, N)) if N == 0 else np.asarray(prob.jac, dtype=np.float64).reshape(len(vert), dim, N)
    dg = None if prob.dg_vert is None else np.asarray(prob.dg_vert, dtype=np.float64).reshape(len(vert), N)
    loss = 0.0
    grad = np.zeros(N)
    for ei, e in enumerate(elem):
        if not m[ei]:
            continue
        d = g[e] - ub[e]
        meas, dmeas = _measure_and_gradient(vert[e])
        q = _mean_half_square(d)
        loss += meas * q
        # the element's measure moves with its vertices: sum_a (d|e|/dv_a) . J_a
        for a in range(dim):
            grad += q * (dmeas[a] @ jac[e[a]])
        # the data moves with theta: |e| int w_a (g - ub) (mean over e) times dg_a/dtheta
        if dg is not None:
            for a in range(dim):
                wa = 0.0
                for b in range(dim):
                    exps = [0] * dim
                    exps[a] += 1
                    exps[b] += 1
                    wa += d[b] * _simplex_monomial(1.0, exps)
                grad += meas * wa * dg[e[a]]
    return float(loss), grad
