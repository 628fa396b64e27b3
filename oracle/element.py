"""Element tensors by quadrature on the physical element (oracle).

A^K_{i1 i2} = a_K(phi_i1, phi_i2) (eq. (elementmatrix), Section 2.2), with the
integrands of the four test cases of Section 3.3:

  mass        phi_i1 * phi_i2                                   (eq. (mass))
  poisson     grad phi_i1 . grad phi_i2                         (eq. (poisson))
  convection  phi_i1 . (w . grad) phi_i2, w = sum_t w_t phi_t   (eq. (navierstokes))
  elasticity  2 mu eps(phi_i1) : eps(phi_i2) + lambda div phi_i1 div phi_i2
              (Section 3.3 writes the eps:eps term; the lambda term and the 2 mu
              scaling are the standard isotropic form with mu = 1, lambda = 1.25)
  source      the linear form v * f, f = sum_t f_t phi_t (L = v*f*dx of the Poisson
              example in Section 5.5): a rank-1 element tensor b^K_i = int phi_i f

Row index i1 is the test function v, column index i2 the trial function u.
Vector spaces use component-blocked local numbering i = c*n_s + s with
phi_i = psi_s e_c.

Geometry is computed from barycentric coordinates: with M the (d+1)x(d+1) matrix
of rows [1, x_j], lambda(x) solves M^T lambda = [1, x], so grad lambda_j is column
j of rows 1..d of M^{-1}, and |K| = |det M| / d!. No reference element, affine
map, reference tensor or geometry tensor is used.
"""
from __future__ import annotations

import math

import numpy as np

from . import basis, quadrature

MASS, POISSON, NS_CONVECTION, ELASTICITY, SOURCE = 0, 1, 2, 3, 4


def integrand_degree(form: int, q: int) -> int:
    if form in (MASS, SOURCE):
        return 2 * q
    if form in (POISSON, ELASTICITY):
        return max(0, 2 * q - 2)
    if form == NS_CONVECTION:
        return 3 * q - 1  # v (q) * w (q) * grad u (q-1)
    raise ValueError(form)


def barycentric_geometry(verts: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """verts [E, d+1, d] -> grad lambda [E, d+1, d] and volume [E]."""
    E, dp1, d = verts.shape
    M = np.concatenate([np.ones((E, dp1, 1)), verts], axis=2)
    Minv = np.linalg.inv(M)
    grad_lam = np.transpose(Minv[:, 1:, :], (0, 2, 1))
    vol = np.abs(np.linalg.det(M)) / math.factorial(d)
    return grad_lam, vol


def _scalar_tables(d: int, q: int, p: int, extra: int):
    lam, w = quadrature.simplex_rule(d, p, extra)
    phi = basis.values(d, q, lam)  # [N, n]
    dphi = basis.bary_derivatives(d, q, lam)  # [N, n, d+1]
    return w, phi, dphi


def _vectorise(d: int, phi: np.ndarray, grad: np.ndarray | None):
    """Component-blocked vector basis from scalar values [N, ns] and gradients [E, N, ns, d]."""
    N, ns = phi.shape
    Phi = np.zeros((N, d * ns, d))
    for c in range(d):
        Phi[:, c * ns:(c + 1) * ns, c] = phi
    if grad is None:
        return Phi, None
    E = grad.shape[0]
    G = np.zeros((E, N, d * ns, d, d))  # [..., component, derivative]
    for c in range(d):
        G[:, :, c * ns:(c + 1) * ns, c, :] = grad
    return Phi, G


def element_tensors(form: int, verts: np.ndarray, q: int, coeffs: np.ndarray | None = None,
                    mu: float = 1.0, lmbda: float = 1.25, extra_points: int = 0,
                    chunk: int | None = None) -> np.ndarray:
    """Element tensors [E, n, n] (bilinear forms) or [E, n] (the source form) in float64
    for cells verts [E, d+1, d]."""
    verts = np.asarray(verts, dtype=np.float64)
    E, dp1, d = verts.shape
    p = integrand_degree(form, q)
    w, phi, dphi = _scalar_tables(d, q, p, extra_points)
    ns = phi.shape[1]
    n = ns if form in (MASS, POISSON, SOURCE) else d * ns
    out = np.empty((E, n)) if form == SOURCE else np.empty((E, n, n))
    if chunk is None:
        per_elem = w.size * n * d * d * 8 * 4
        chunk = max(1, min(E, int(64e6 // max(per_elem, 1))))
    for s in range(0, E, chunk):
        v = verts[s:s + chunk]
        grad_lam, vol = barycentric_geometry(v)
        if form == MASS:
            local = np.einsum("q,qi,qj->ij", w, phi, phi, optimize=True)
            out[s:s + chunk] = vol[:, None, None] * local[None]
            continue
        if form == SOURCE:
            f = np.einsum("et,qt->eq", np.asarray(coeffs[s:s + chunk], dtype=np.float64), phi, optimize=True)
            out[s:s + chunk] = vol[:, None] * np.einsum("q,qi,eq->ei", w, phi, f, optimize=True)
            continue
        grad = np.einsum("qij,ejb->eqib", dphi, grad_lam)  # [e, q, ns, d]
        if form == POISSON:
            out[s:s + chunk] = vol[:, None, None] * np.einsum("q,eqib,eqjb->eij", w, grad, grad, optimize=True)
        elif form == NS_CONVECTION:
            Phi, G = _vectorise(d, phi, grad)
            c = np.asarray(coeffs[s:s + chunk], dtype=np.float64)  # [e, n]
            wq = np.einsum("et,qtc->eqc", c, Phi, optimize=True)  # w(x_q)
            conv = np.einsum("eqb,eqjcb->eqjc", wq, G, optimize=True)  # (w . grad) phi_j
            out[s:s + chunk] = vol[:, None, None] * np.einsum("q,qic,eqjc->eij", w, Phi, conv, optimize=True)
        elif form == ELASTICITY:
            _, G = _vectorise(d, phi, grad)
            eps = 0.5 * (G + np.swapaxes(G, -1, -2))
            div = np.trace(G, axis1=-2, axis2=-1)
            a = 2.0 * mu * np.einsum("q,eqirs,eqjrs->eij", w, eps, eps, optimize=True)
            a += lmbda * np.einsum("q,eqi,eqj->eij", w, div, div, optimize=True)
            out[s:s + chunk] = vol[:, None, None] * a
        else:
            raise ValueError(form)
    return out


def frobenius_rel_error(A: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-element ||A - ref||_F / ||ref||_F (absolute error where ||ref||_F = 0)."""
    A = A.reshape(A.shape[0], -1).astype(np.float64)
    ref = ref.reshape(ref.shape[0], -1).astype(np.float64)
    num = np.linalg.norm(A - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
