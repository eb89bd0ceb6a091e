"""Plain FP64 estimators over per-walk oracle outputs (test infrastructure only).

Walk (p, w) of a run sits at row p * W + w.  Each function is the textbook
definition of the quantity, written out without blocking or fusion.
"""
from __future__ import annotations

import numpy as np


def point_mean_se(values: np.ndarray, n_points: int, W: int):
    """Per-point sample mean and standard error of the mean (ddof = 1)."""
    v = np.asarray(values, dtype=np.float64).reshape((n_points, W) + np.shape(values)[1:])
    mean = v.mean(axis=1)
    se = v.std(axis=1, ddof=1) / np.sqrt(W) if W > 1 else np.zeros_like(mean)
    return mean, se


def ustat_product(u: np.ndarray, udot: np.ndarray) -> np.ndarray:
    """Eq. (ustatistics): sum_m udot_m (S - u_m) / (n (n - 1)), S = sum_m u_m."""
    u = np.asarray(u, dtype=np.float64)
    udot = np.asarray(udot, dtype=np.float64)
    n = u.shape[0]
    S = u.sum()
    return (udot * (S - u).reshape((n,) + (1,) * (udot.ndim - 1))).sum(axis=0) / (n * (n - 1))


def grad_l2_ustat(u_hat, udot, u_ref, n_points: int, W: int, B: int) -> np.ndarray:
    """Gradient of L = 1/2 sum_p (u_p - uref_p)^2 (Eq. squared_loss_deriv), with
    the product u * udot from the U-statistic estimator applied in batches of B
    consecutive walks (Sec. 4.3; B = 8 in Sec. 5.3).  Per point: the mean over
    batches of  sum_m udot_m [(S - u_m)/(B(B-1)) - uref/B];  summed over points."""
    if W % B:
        raise ValueError("walks per point must be a multiple of B")
    N = np.shape(udot)[1]
    nb = W // B
    u = np.asarray(u_hat, dtype=np.float64).reshape(n_points, nb, B)
    ud = np.asarray(udot, dtype=np.float64).reshape(n_points, nb, B, N)
    ur = np.asarray(u_ref, dtype=np.float64).reshape(n_points, 1)
    total = np.zeros(N)
    for p in range(n_points):
        acc = np.zeros(N)
        for b in range(nb):
            acc += ustat_product(u[p, b], ud[p, b]) - ur[p, 0] * ud[p, b].mean(axis=0)
        total += acc / nb
    return total


def grad_l2_uncorrelated(u_hat, udot, u_ref, n_points: int, W: int) -> np.ndarray:
    """Eq. (uncorrelated_product): u from walks 1..M, udot from walks M+1..2M."""
    M = W // 2
    u = np.asarray(u_hat, dtype=np.float64).reshape(n_points, W)
    ud = np.asarray(udot, dtype=np.float64).reshape(n_points, W, -1)
    ubar = u[:, :M].mean(axis=1)
    udbar = ud[:, M:2 * M].mean(axis=1)
    return ((ubar - np.asarray(u_ref))[:, None] * udbar).sum(axis=0)


def grad_l2_correlated(u_hat, udot, u_ref, n_points: int, W: int) -> np.ndarray:
    """Eq. (correlated_product): both means over all walks (biased)."""
    u = np.asarray(u_hat, dtype=np.float64).reshape(n_points, W)
    ud = np.asarray(udot, dtype=np.float64).reshape(n_points, W, -1)
    return ((u.mean(axis=1) - np.asarray(u_ref))[:, None] * ud.mean(axis=1)).sum(axis=0)


def vjp(udot, w, n_points: int, W: int) -> np.ndarray:
    """sum_p w_p E[udot_p] with the plain per-point mean."""
    ud = np.asarray(udot, dtype=np.float64).reshape(n_points, W, -1)
    return (np.asarray(w, dtype=np.float64)[:, None] * ud.mean(axis=1)).sum(axis=0)


def loss_l2(u_hat, u_ref, n_points: int, W: int) -> float:
    u = np.asarray(u_hat, dtype=np.float64).reshape(n_points, W).mean(axis=1)
    return 0.5 * float(((u - np.asarray(u_ref)) ** 2).sum())
