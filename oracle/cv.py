"""The nested walks' control-variate table, in FP64 (test infrastructure only).

Each nested walk launched from x_off = xbar - h n contributes
u - (q n + t) . (x_end - x_off) to the backward difference of Eq.
(dudn_fd_estimate); per boundary element the table holds (q, t): q a surrogate
of du/dn and t the tangential gradient of the Dirichlet data on the element.
For data given per vertex and interpolated linearly, t is the gradient of the
interpolant along the element: the vector in the span of the element's edges
e_i = v_i - v_0 with t . e_i = g_i - g_0 (i = 1 for a segment, 1 and 2 for a
triangle), i.e. t = E^T (E E^T)^-1 r with E the edge rows and r the value
differences.  Only the tests use this module.
"""
from __future__ import annotations

import numpy as np


def tangential_gradient(vert: np.ndarray, elem: np.ndarray, g_vert: np.ndarray) -> np.ndarray:
    """(n_elem, 3): the data's gradient along each element (third column 0 in 2D)."""
    v = np.asarray(vert, dtype=np.float64)
    g = np.asarray(g_vert, dtype=np.float64)
    elem = np.asarray(elem)
    k = elem.shape[1] - 1                                   # edges per element: 1 or 2
    E = np.stack([v[elem[:, i]] - v[elem[:, 0]] for i in range(1, k + 1)], axis=1)   # (m, k, dim)
    r = np.stack([g[elem[:, i]] - g[elem[:, 0]] for i in range(1, k + 1)], axis=1)   # (m, k)
    gram = np.einsum("mid,mjd->mij", E, E)
    coef = np.linalg.solve(gram, r[:, :, None])[:, :, 0]                          # (m, k)
    t = np.einsum("mi,mid->md", coef, E)
    out = np.zeros((elem.shape[0], 3))
    out[:, :v.shape[1]] = t
    return out


def nested_cv_table(vert: np.ndarray, elem: np.ndarray, g_vert: np.ndarray, q) -> np.ndarray:
    """(n_elem, 4) float32 table (q, t0, t1, t2) for the nested walks' correction."""
    tab = np.zeros((np.asarray(elem).shape[0], 4), dtype=np.float32)
    tab[:, 0] = np.asarray(q, dtype=np.float64)
    tab[:, 1:] = tangential_gradient(vert, elem, g_vert)
    return tab
