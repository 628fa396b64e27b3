"""Pins of the curved-cell oracle (quadrature representation, Section 3.4) against facts
other than itself:

* the collapsed Gauss-Jacobi rule integrates monomials over the reference simplex exactly
  (closed form prod(alpha_a!) / (|alpha| + d)!) up to its degree, and its weights sum to
  the simplex's measure 1/d!;
* on straight cells, for any geometry degree, the element tensors equal the affine
  oracle's (already pinned against exact rationals and the paper's printed values);
* on cells mapped by a quadratic map with a closed-form Jacobian determinant, the sum
  of the mass matrix is the cell's exact area / volume;
* on curved cells, identities that hold for every quadrature rule: the Poisson rows sum
  to zero (the basis sums to one), and for P2 on quadratic geometry the coordinate
  function x_0 is in the space, so u^T A u with u its nodal values equals the rule's
  measure of the cell (|grad x_0| = 1), i.e. the sum of the mass matrix;
* a planted mistake (grad_x phi formed with F'^-1 instead of F'^-T) breaks the last
  identity, so it would catch that transpose.
"""
import math

import numpy as np
import pytest

from oracle import basis
from oracle import curved as OC
from oracle import element as OE
from synthetic import mesh as M
from synthetic.curved import curved_mesh, gather_nodes


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("p", [0, 1, 3, 4, 7])
def test_collapsed_rule_is_exact_for_monomials(d, p):
    X, w = OC.collapsed_rule(d, p)
    assert abs(w.sum() - 1.0 / math.factorial(d)) < 1e-15
    m = max(1, math.ceil((p + 1) / 2))
    assert X.shape[0] == m ** d
    for alpha in np.ndindex(*([p + 1] * d)):
        if sum(alpha) > p:
            continue
        exact = np.prod([math.factorial(a) for a in alpha]) / math.factorial(sum(alpha) + d)
        got = float(np.sum(w * np.prod(X ** np.array(alpha)[None, :], axis=1)))
        assert abs(got - exact) <= 1e-15 * max(1.0, exact) + 1e-17


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("form", [OC.MASS, OC.POISSON])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_straight_cells_equal_the_affine_oracle(d, form, q):
    m = M.unit_square_triangles(3, 0.25, 11) if d == 2 else M.unit_cube_tets(2, 0.25, 11)
    V = M.gather_cell_vertices(m)
    ref = OE.element_tensors(form, V, q)
    for g in (1, 2):
        got = OC.element_tensors_curved(form, OC.affine_nodes(V, g), q, g, 2 * q)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _mapped_reference_cell(d, c):
    """P2 nodes of the reference simplex moved by a quadratic map whose Jacobian
    determinant is affine: 2D F = (X_0, X_1 + c X_0 X_1), det F' = 1 + c X_0;
    3D F = (X_0 (1 + c X_1), X_1, X_2), det F' = 1 + c X_1."""
    lat = np.array(basis.lattice(d, 2), dtype=float) / 2  # barycentric [n_g, d+1]
    X = lat[:, 1:]  # reference coordinates of the P2 nodes
    F = X.copy()
    if d == 2:
        F[:, 1] = X[:, 1] + c * X[:, 0] * X[:, 1]  # det = 1 + c X_0
    else:
        F[:, 0] = X[:, 0] * (1.0 + c * X[:, 1])    # det = 1 + c X_1
    return F


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_mass_sum_is_the_exact_measure_of_a_mapped_cell(d, q):
    c = 0.7
    nodes = _mapped_reference_cell(d, c)[None]
    # area 1/2 + c * int X_0 = 1/2 + c/6; volume 1/6 + c * int X_1 = 1/6 + c/24
    exact = 0.5 + c / 6.0 if d == 2 else 1.0 / 6.0 + c / 24.0
    A = OC.element_tensors_curved(OC.MASS, nodes, q, 2, 2 * q + d)
    assert abs(A.sum() - exact) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_curved_poisson_identities(d):
    cm = curved_mesh(d, 2 if d == 3 else 3, eps=0.12)
    X = gather_nodes(cm)
    p = 7
    A = OC.element_tensors_curved(OC.POISSON, X, 2, 2, p)
    Mm = OC.element_tensors_curved(OC.MASS, X, 2, 2, p)
    assert np.abs(A.sum(axis=2)).max() <= 1e-13 * np.abs(A).max()
    for a in range(d):
        u = X[:, :, a]  # nodal values of the coordinate x_a (P2 nodes = geometry nodes)
        energy = np.einsum("ei,eij,ej->e", u, A, u)
        assert np.abs(energy - Mm.sum(axis=(1, 2))).max() <= 1e-13
    # the cells really are curved: the rule's measure differs from the straight cells'
    straight = OC.element_tensors_curved(OC.MASS, OC.affine_nodes(X[:, :d + 1], 1), 2, 1, p).sum(axis=(1, 2))
    assert np.abs(Mm.sum(axis=(1, 2)) - straight).max() > 1e-4


def test_a_transposed_inverse_breaks_the_energy_identity():
    cm = curved_mesh(2, 3, eps=0.12)
    X = gather_nodes(cm)
    Xq, w = OC.collapsed_rule(2, 7)
    dg = OC.reference_gradients(2, 2, Xq)
    dphi = OC.reference_gradients(2, 2, Xq)
    bad = np.zeros((X.shape[0], 6, 6))
    for k in range(Xq.shape[0]):
        J = np.einsum("ena,nb->eab", X, dg[k])
        Jinv = np.linalg.inv(J)
        gx = np.einsum("eab,nb->ena", Jinv, dphi[k])  # planted: F'^-1 instead of F'^-T
        bad += w[k] * np.abs(np.linalg.det(J))[:, None, None] * np.einsum("eia,eja->eij", gx, gx)
    Mm = OC.element_tensors_curved(OC.MASS, X, 2, 2, 7).sum(axis=(1, 2))
    u = X[:, :, 0]
    energy = np.einsum("ei,eij,ej->e", u, bad, u)
    assert np.abs(energy - Mm).max() > 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_curved_p3_energy_identity(d):
    """P3 on quadratic-geometry cells: the coordinate x_a is a quadratic function of X, so
    it lies in the P3 space and its nodal interpolant (values of the map at the P3
    lattice points) is exact; u^T A u is then the rule's measure of the cell, the sum of
    the P3 mass matrix (which sums the P3 basis, a partition of unity)."""
    cm = curved_mesh(d, 2 if d == 3 else 3, eps=0.12)
    X = gather_nodes(cm)  # [E, n_g, d], P2 geometry nodes
    p = 9
    A = OC.element_tensors_curved(OC.POISSON, X, 3, 2, p)
    Mm = OC.element_tensors_curved(OC.MASS, X, 3, 2, p)
    lat3 = np.array(basis.lattice(d, 3), dtype=float) / 3  # barycentric P3 lattice [n3, d+1]
    psi2 = basis.values(d, 2, lat3)  # the geometry basis at the P3 lattice points [n3, n_g]
    x3 = np.einsum("sn,ena->esa", psi2, X)  # the map at the P3 nodes [E, n3, d]
    assert np.abs(A.sum(axis=2)).max() <= 1e-13 * np.abs(A).max()
    for a in range(d):
        u = x3[:, :, a]
        energy = np.einsum("ei,eij,ej->e", u, A, u)
        assert np.abs(energy - Mm.sum(axis=(1, 2))).max() <= 1e-13
