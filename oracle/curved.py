"""Element tensors of the mass and Poisson forms on curved simplices by quadrature
(oracle; test infrastructure only).

Section 3.4 ("Curvilinear elements"): when the map F_K from the reference simplex K0 to
the cell is not affine, its Jacobian varies inside the cell; the element tensor is then
approximated by a quadrature sum over reference points X_k with weights w_k,

    A^K_{i1 i2} ~= sum_k w_k f_{i1 i2}(X_k) |det F_K'(X_k)|,
    mass     f = Phi_i1 Phi_i2
    Poisson  f = grad_x phi_i1 . grad_x phi_i2,  grad_x phi = F_K'^{-T} grad_X Phi.

This module evaluates that sum as written, point by point: the physical gradients are
formed explicitly at every point; no reference tensor with a point index and no
geometry tensor is built.

The map is the geometry interpolant F_K(X) = sum_n x_n Psi_n(X) of degree g over the
cell's nodes x_n, given in the local dof order of the P_g Lagrange space (g = 1: the
vertices, an affine map; g = 2: vertices then edge nodes, a quadratic map), so
F_K'(X)[a][b] = sum_n x_n[a] dPsi_n/dX_b(X).

The rule is the collapsed (conical product) Gauss-Jacobi rule of Karniadakis and
Sherwin, "Spectral/hp Element Methods", with m points per direction: direction k
(k = 0, ..., d-1) takes the m-point Gauss-Jacobi rule on [0, 1] for the weight
(1 - u)^k (the Jacobian of the collapse absorbed into the weight), the point is
X_k = u_k prod_{l > k} (1 - u_l), the weight the product of the directions' weights. It is
exact for polynomials of degree 2m - 1 on K0, and m = ceil((p + 1) / 2) for degree p.
The 1-D rules are scipy.special.roots_jacobi (weight (1 - x)^a (1 + x)^b on [-1, 1]).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import roots_jacobi

from . import basis

MASS, POISSON = 0, 1


def gauss_jacobi01(m: int, a: float) -> tuple[np.ndarray, np.ndarray]:
    """m-point Gauss-Jacobi rule on [0, 1] for the weight (1 - u)^a."""
    x, w = roots_jacobi(m, a, 0.0)
    return 0.5 * (1.0 + x), w / 2.0 ** (a + 1.0)


def collapsed_rule(d: int, p: int) -> tuple[np.ndarray, np.ndarray]:
    """Reference points X [N, d] and weights [N] (summing to 1/d!), exact for degree p."""
    m = max(1, math.ceil((p + 1) / 2))
    rules = [gauss_jacobi01(m, float(k)) for k in range(d)]
    grids = np.meshgrid(*[r[0] for r in rules], indexing="ij")
    wgrids = np.meshgrid(*[r[1] for r in rules], indexing="ij")
    U = np.stack([g.reshape(-1) for g in grids], axis=1)
    W = np.prod(np.stack([g.reshape(-1) for g in wgrids], axis=1), axis=1)
    X = np.empty_like(U)
    for k in range(d):
        v = U[:, k].copy()
        for l in range(k + 1, d):
            v = v * (1.0 - U[:, l])
        X[:, k] = v
    return X, W


def _bary(X: np.ndarray) -> np.ndarray:
    return np.concatenate([(1.0 - X.sum(axis=1))[:, None], X], axis=1)


def reference_gradients(d: int, q: int, X: np.ndarray) -> np.ndarray:
    """dPhi/dX at reference points X [N, d] -> [N, n, d] (chain rule through lambda)."""
    dl = basis.bary_derivatives(d, q, _bary(X))  # [N, n, d+1]
    return dl[:, :, 1:] - dl[:, :, :1]


def element_tensors_curved(form: int, nodes: np.ndarray, q: int, g: int, p: int) -> np.ndarray:
    """nodes [E, n_g, d] (the cells' geometry nodes, P_g local order) -> A^K [E, n, n] by the
    degree-p collapsed Gauss-Jacobi rule."""
    E, ng, d = nodes.shape
    X, w = collapsed_rule(d, p)
    dpsi_geo = reference_gradients(d, g, X)  # [N, n_g, d]
    if dpsi_geo.shape[1] != ng:
        raise ValueError("nodes do not match the geometry degree")
    phi = basis.values(d, q, _bary(X))  # [N, n]
    dphi = reference_gradients(d, q, X)  # [N, n, d]
    n = phi.shape[1]
    out = np.zeros((E, n, n))
    for k in range(X.shape[0]):
        J = np.einsum("ena,nb->eab", nodes, dpsi_geo[k])  # [E, d, d], J[a][b] = dx_a/dX_b
        det = np.abs(np.linalg.det(J))
        if form == MASS:
            out += w[k] * det[:, None, None] * np.outer(phi[k], phi[k])[None]
        elif form == POISSON:
            Jinv = np.linalg.inv(J)  # [E, d, d]
            gx = np.einsum("eba,nb->ena", Jinv, dphi[k])  # grad_x phi = J^{-T} grad_X Phi
            out += w[k] * det[:, None, None] * np.einsum("eia,eja->eij", gx, gx)
        else:
            raise ValueError(form)
    return out


def affine_nodes(vertices: np.ndarray, g: int) -> np.ndarray:
    """The P_g lattice nodes of straight cells: vertices [E, d+1, d] -> [E, n_g, d]
    (barycentric combinations of the vertices in the local dof order)."""
    d = vertices.shape[2]
    lat = np.array(basis.lattice(d, g), dtype=float) / g  # [n_g, d+1]
    return np.einsum("sj,ejx->esx", lat, vertices)
