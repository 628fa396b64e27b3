"""Quadrature for the oracle: Gauss-Legendre on [-1, 1] and a collapsed (Duffy) rule
on the reference simplex, returned in barycentric coordinates so that it transfers
to any physical simplex by scaling the weights with the simplex volume.

The paper integrates with collapsed Gauss-Jacobi rules (Section 6); the oracle
deliberately uses Gauss-Legendre with the Duffy Jacobian folded into the weights,
a different rule that is exact for the same polynomial degrees.

Exactness: with m points per direction Gauss-Legendre integrates degree 2m-1.
The collapse (X_1, ..., X_d) = (u_1 (1-u_2)...(1-u_d), ..., u_d) with Jacobian
prod_k (1-u_k)^(k-1) raises the degree in u_d by d-1, so a degree-p integrand
needs m = ceil((p + d) / 2).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(m: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes and weights of the m-point Gauss-Legendre rule on [-1, 1].

    Newton iteration on P_m, evaluated by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; P_m' = m (x P_m - P_{m-1}) / (x^2 - 1).
    """
    x = np.cos(np.pi * (np.arange(m) + 0.75) / (m + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(1, m):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        if m == 0:
            raise ValueError("m >= 1")
        dp = m * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(1, m):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = m * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def points_for_degree(p: int, d: int) -> int:
    return max(1, math.ceil((p + d) / 2))


def simplex_rule(d: int, p: int, extra: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Barycentric points [N, d+1] and weights [N] (summing to 1) exact for degree p.

    ``extra`` adds points per direction (used for brute-force checks)."""
    m = points_for_degree(p, d) + extra
    t, wt = gauss_legendre(m)
    u = 0.5 * (t + 1.0)
    wu = 0.5 * wt
    grids = np.meshgrid(*([u] * d), indexing="ij")
    wgrids = np.meshgrid(*([wu] * d), indexing="ij")
    U = np.stack([g.reshape(-1) for g in grids], axis=1)  # [N, d], U[:, 0] = u_1 ...
    W = np.prod(np.stack([g.reshape(-1) for g in wgrids], axis=1), axis=1)
    X = np.empty_like(U)
    jac = np.ones(U.shape[0])
    # X_k = u_k * prod_{l>k} (1 - u_l); Jacobian prod_l (1 - u_l)^(l-1) (l counted from 1)
    for k in range(d):
        v = U[:, k].copy()
        for l in range(k + 1, d):
            v = v * (1.0 - U[:, l])
        X[:, k] = v
    for l in range(1, d):
        jac = jac * (1.0 - U[:, l]) ** l
    W = W * jac
    lam = np.concatenate([(1.0 - X.sum(axis=1))[:, None], X], axis=1)
    # the reference simplex has measure 1/d!; normalise so the weights sum to 1
    return lam, W * math.factorial(d)
