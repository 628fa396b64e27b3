"""Lagrange P_q basis on a d-simplex in barycentric coordinates (oracle).

The basis function attached to the lattice point with barycentric multi-index k
(|k| = q, Section 5.3 of the paper: Lagrange elements, nodes given by point
evaluation at the equispaced lattice) is Silvester's product

    phi_k(lambda) = prod_j prod_{m=0}^{k_j-1} (q*lambda_j - m) / (m + 1),

which is 1 at its own lattice point and 0 at every other one. Derivatives with
respect to lambda_j follow from the product rule.

Local dof order (shared convention, implemented separately here): for
m = 0..d, for each vertex subset S of size m+1 in lexicographic order, the lattice
points whose support is exactly S, in descending lexicographic order of k.
Vertices first, then edges (01, 02, 03, 12, 13, 23), faces, interior.
"""
from __future__ import annotations

import itertools

import numpy as np


def lattice(d: int, q: int) -> list[tuple[int, ...]]:
    pts_all = [k for k in itertools.product(range(q + 1), repeat=d + 1) if sum(k) == q]
    order = []
    for m in range(d + 1):
        for subset in itertools.combinations(range(d + 1), m + 1):
            pts = [k for k in pts_all if tuple(j for j in range(d + 1) if k[j] > 0) == subset]
            order.extend(sorted(pts, reverse=True))
    return order


def _factor(q: int, kj: int, lam: np.ndarray) -> np.ndarray:
    """prod_{m<kj} (q*lam - m)/(m+1) for one barycentric coordinate."""
    out = np.ones_like(lam)
    for m in range(kj):
        out = out * (q * lam - m) / (m + 1)
    return out


def _factor_derivative(q: int, kj: int, lam: np.ndarray) -> np.ndarray:
    """d/dlam of _factor by the product rule."""
    out = np.zeros_like(lam)
    for skip in range(kj):
        term = np.full_like(lam, q / (skip + 1))
        for m in range(kj):
            if m != skip:
                term = term * (q * lam - m) / (m + 1)
        out = out + term
    return out


def values(d: int, q: int, lam: np.ndarray) -> np.ndarray:
    """phi_k at barycentric points lam [N, d+1] -> [N, n]."""
    ks = lattice(d, q)
    out = np.empty((lam.shape[0], len(ks)))
    for i, k in enumerate(ks):
        v = np.ones(lam.shape[0])
        for j in range(d + 1):
            v = v * _factor(q, k[j], lam[:, j])
        out[:, i] = v
    return out


def bary_derivatives(d: int, q: int, lam: np.ndarray) -> np.ndarray:
    """d phi_k / d lambda_j at lam [N, d+1] -> [N, n, d+1] (lambda_j treated as independent)."""
    ks = lattice(d, q)
    out = np.empty((lam.shape[0], len(ks), d + 1))
    for i, k in enumerate(ks):
        f = [_factor(q, k[j], lam[:, j]) for j in range(d + 1)]
        for jd in range(d + 1):
            v = _factor_derivative(q, k[jd], lam[:, jd])
            for j in range(d + 1):
                if j != jd:
                    v = v * f[j]
            out[:, i, jd] = v
    return out
