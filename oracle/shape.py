"""Shape derivative of L(x) = u^T A(x) v for the Poisson form (oracle).

A(x) is the assembled Poisson matrix (eq. (poisson), Section 3.3) of the mesh with
vertex coordinates x; u, v are fixed coefficient vectors, so u_h = sum u_i phi_i
and v_h move with the mesh. For a velocity field V the continuous shape
derivative of L = int grad u_h . grad v_h is

    dL[V] = sum_K int_K (div V) grad u_h . grad v_h - grad u_h . (DV + DV^T) grad v_h dx,

exact for Lagrange functions transported by a piecewise-affine V. Taking V the
hat function of vertex k times e_c (on cell K: V = lambda_j e_c, j the local index
of k) gives dL/dx_{k,c}:

    sum_{K ∋ k} int_K d_c lambda_j (gu . gv) - d_c u (grad lambda_j . gv)
                       - (gu . grad lambda_j) d_c v dx.

The integrals are evaluated with the oracle's quadrature on each physical cell.
"""
from __future__ import annotations

import numpy as np

from . import basis, quadrature
from .element import barycentric_geometry


def poisson_objective(verts_all: np.ndarray, cells: np.ndarray, q: int, dofmap: np.ndarray,
                      u: np.ndarray, v: np.ndarray) -> float:
    """L = u^T A v evaluated cell by cell (sum_K u_K^T A^K v_K)."""
    from .element import POISSON, element_tensors

    A = element_tensors(POISSON, verts_all[cells], q)
    uK = u[dofmap]
    vK = v[dofmap]
    return float(np.einsum("ei,eij,ej->", uK, A, vK))


def poisson_shape_gradient(verts_all: np.ndarray, cells: np.ndarray, q: int, dofmap: np.ndarray,
                           u: np.ndarray, v: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """dL/dx [n_v, d] for L = u^T A(x) v, Poisson P_q."""
    n_v, d = verts_all.shape
    lam, w = quadrature.simplex_rule(d, max(0, 2 * q - 2))
    dphi = basis.bary_derivatives(d, q, lam)
    out = np.zeros((n_v, d))
    E = cells.shape[0]
    for s in range(0, E, chunk):
        c = cells[s:s + chunk]
        grad_lam, vol = barycentric_geometry(verts_all[c])
        grad = np.einsum("qij,ejb->eqib", dphi, grad_lam)
        gu = np.einsum("ei,eqib->eqb", u[dofmap[s:s + chunk]], grad)
        gv = np.einsum("ei,eqib->eqb", v[dofmap[s:s + chunk]], grad)
        uv = np.einsum("q,eqb,eqb->e", w, gu, gv)
        t1 = grad_lam * uv[:, None, None]
        t2 = np.einsum("q,eqc,ejb,eqb->ejc", w, gu, grad_lam, gv)
        t3 = np.einsum("q,eqb,ejb,eqc->ejc", w, gu, grad_lam, gv)
        contrib = vol[:, None, None] * (t1 - t2 - t3)
        np.add.at(out, c, contrib)
    return out
