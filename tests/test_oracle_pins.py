"""Pins of the CPU oracle against facts fixed by the paper and by mathematics:
library routines, closed forms, printed values, exact rational arithmetic and
invariants. None of these compares the oracle with itself."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import exact_forms as X
from oracle import basis, element, quadrature
from oracle.element import ELASTICITY, MASS, NS_CONVECTION, POISSON
from synthetic.dofmap import local_lattice, n_local

HERE = os.path.dirname(os.path.abspath(__file__))
RNG = np.random.default_rng(12345)


def random_simplices(d, E, rng=RNG):
    """Well-shaped random simplices: a jittered reference simplex, scaled and moved."""
    ref = np.vstack([np.zeros(d), np.eye(d)])
    v = ref[None] + rng.uniform(-0.2, 0.2, size=(E, d + 1, d))
    v = v * rng.uniform(0.05, 2.0, size=(E, 1, 1)) + rng.uniform(-3, 3, size=(E, 1, d))
    return v


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 12])
def test_gauss_legendre_matches_numpy(m):
    x, w = quadrature.gauss_legendre(m)
    xr, wr = np.polynomial.legendre.leggauss(m)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("p", [0, 1, 2, 5, 8])
def test_simplex_rule_integrates_moments(d, p):
    lam, w = quadrature.simplex_rule(d, p)
    Xp = lam[:, 1:]
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(lam.sum(axis=1), 1.0)
    for a in X.monomials(d, p):
        got = np.sum(w * np.prod(Xp ** np.array(a), axis=1)) / math.factorial(d)
        assert abs(got - float(X.moment(a))) < 1e-15 + 1e-13 * float(X.moment(a))


def test_simplex_rule_is_not_exact_beyond_its_degree():
    # a degree-(2m) monomial in the last collapsed direction breaks an m-point rule
    d, p = 3, 3
    lam, w = quadrature.simplex_rule(d, p)
    m = quadrature.points_for_degree(p, d)
    a = (0, 0, 2 * m)
    got = np.sum(w * lam[:, 3] ** a[2]) / 6
    assert abs(got - float(X.moment(a))) > 1e-8


# ---------------------------------------------------------------- basis
@pytest.mark.parametrize("d,q", [(2, 1), (2, 3), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_basis_is_nodal_and_a_partition_of_unity(d, q):
    ks = basis.lattice(d, q)
    assert len(ks) == n_local(d, q)
    assert [tuple(k) for k in local_lattice(d, q)] == ks  # same order as the dofmap builder
    nodes = np.array(ks, dtype=float) / q
    V = basis.values(d, q, nodes)
    assert np.allclose(V, np.eye(len(ks)), atol=1e-14)
    lam = quadrature.simplex_rule(d, 4)[0]
    assert np.allclose(basis.values(d, q, lam).sum(axis=1), 1.0, atol=1e-13)


@pytest.mark.parametrize("d,q", [(2, 3), (3, 4)])
def test_basis_barycentric_derivatives_vs_finite_differences(d, q):
    lam = quadrature.simplex_rule(d, 3)[0]
    D = basis.bary_derivatives(d, q, lam)
    h = 1e-6
    for j in range(d + 1):
        lp = lam.copy(); lp[:, j] += h
        lm = lam.copy(); lm[:, j] -= h
        fd = (basis.values(d, q, lp) - basis.values(d, q, lm)) / (2 * h)
        assert np.allclose(D[:, :, j], fd, atol=1e-7 * q**q)


def test_p3_triangle_local_order_puts_vertices_first_and_bubble_last():
    ks = basis.lattice(2, 3)
    assert ks[:3] == [(3, 0, 0), (0, 3, 0), (0, 0, 3)]
    assert ks[9] == (1, 1, 1)


# ---------------------------------------------------------------- printed values
def test_p3_triangle_poisson_printed_entries():
    rows = np.loadtxt(os.path.join(HERE, "golden", "p3_triangle_poisson.txt"))
    for r in rows:
        v = r[:6].reshape(1, 3, 2)
        A = element.element_tensors(POISSON, v, 3)[0]
        got = [A[0, 0], A[0, 1], A[0, 2], A[9, 9]]
        assert np.allclose(got, r[6:], atol=1e-13, rtol=0)


# ---------------------------------------------------------------- closed forms
def test_p1_triangle_laplacian_reference_and_cotangent_formula():
    ref = np.array([[[0, 0], [1, 0], [0, 1]]], float)
    A = element.element_tensors(POISSON, ref, 1)[0]
    assert np.allclose(A, [[1, -.5, -.5], [-.5, .5, 0], [-.5, 0, .5]], atol=1e-15)
    v = random_simplices(2, 50)
    A = element.element_tensors(POISSON, v, 1)
    for e in range(50):
        P = v[e]
        for i in range(3):
            for j in range(3):
                if i == j:
                    continue
                k = 3 - i - j
                a, b = P[i] - P[k], P[j] - P[k]
                cot = np.dot(a, b) / abs(a[0] * b[1] - a[1] * b[0])
                assert abs(A[e, i, j] - (-0.5 * cot)) < 1e-12 * max(1, abs(cot))
        assert np.allclose(A[e].sum(axis=1), 0, atol=1e-13)


def test_p1_mass_closed_forms():
    v2 = random_simplices(2, 20)
    a, b = v2[:, 1] - v2[:, 0], v2[:, 2] - v2[:, 0]
    area = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    M = element.element_tensors(MASS, v2, 1)
    ref = area[:, None, None] / 12 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])
    assert np.allclose(M, ref, rtol=1e-14, atol=0)
    v3 = random_simplices(3, 20)
    vol = np.abs(np.einsum("ei,ei->e", v3[:, 1] - v3[:, 0],
                           np.cross(v3[:, 2] - v3[:, 0], v3[:, 3] - v3[:, 0]))) / 6
    M = element.element_tensors(MASS, v3, 1)
    ref = vol[:, None, None] / 20 * (np.eye(4) + np.ones((4, 4)))
    assert np.allclose(M, ref, rtol=1e-14, atol=0)


def test_p1_tet_laplacian_from_face_area_vectors():
    v = random_simplices(3, 30)
    A = element.element_tensors(POISSON, v, 1)
    for e in range(30):
        P = v[e]
        vol = abs(np.dot(P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))) / 6
        area = []
        for i in range(4):
            j, k, l = [m for m in range(4) if m != i]
            n = 0.5 * np.cross(P[k] - P[j], P[l] - P[j])
            if np.dot(n, P[j] - P[i]) < 0:
                n = -n  # outward from the face opposite vertex i
            area.append(n)
        # grad lambda_i = -n_i / (3 |K|): A_ij = |K| grad lambda_i . grad lambda_j
        ref = np.array([[np.dot(area[i], area[j]) / (9 * vol) for j in range(4)] for i in range(4)])
        assert np.allclose(A[e], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


# ---------------------------------------------------------------- exact rational
EXACT_CASES = [(MASS, 1), (MASS, 2), (MASS, 3), (POISSON, 1), (POISSON, 2), (POISSON, 3),
               (ELASTICITY, 1), (ELASTICITY, 2)]

RATIONAL_TETS = [
    [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
    [(Fraction(1, 3), 0, 0), (Fraction(1, 2), Fraction(1, 10), 0), (Fraction(1, 5), Fraction(3, 5), Fraction(1, 7)),
     (Fraction(1, 9), Fraction(1, 4), Fraction(2, 3))],
    [(0, 0, 0), (1, 0, 0), (0, 1, 0), (Fraction(1, 2), Fraction(1, 2), Fraction(-3, 4))],  # negative orientation
]


@pytest.mark.parametrize("form,q", EXACT_CASES)
@pytest.mark.parametrize("t", range(len(RATIONAL_TETS)))
def test_element_tensor_vs_exact_rational(form, q, t):
    verts = [tuple(Fraction(c) for c in v) for v in RATIONAL_TETS[t]]
    ref = np.array(X.element_tensor(form, verts, q), dtype=float)
    vf = np.array([[float(c) for c in v] for v in verts])[None]
    A = element.element_tensors(form, vf, q)[0]
    assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("t", range(len(RATIONAL_TETS)))
def test_convection_vs_exact_rational(t):
    verts = [tuple(Fraction(c) for c in v) for v in RATIONAL_TETS[t]]
    w = [Fraction((7 * i) % 11 - 5, 3) for i in range(30)]
    ref = np.array(X.element_tensor(NS_CONVECTION, verts, 2, w=w), dtype=float)
    vf = np.array([[float(c) for c in v] for v in verts])[None]
    A = element.element_tensors(NS_CONVECTION, vf, 2, coeffs=np.array([[float(x) for x in w]]))[0]
    assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()


def test_triangle_p3_poisson_vs_exact_rational():
    verts = [(Fraction(1, 3), Fraction(0)), (Fraction(2), Fraction(1, 5)), (Fraction(1, 2), Fraction(7, 4))]
    ref = np.array(X.element_tensor(POISSON, verts, 3), dtype=float)
    A = element.element_tensors(POISSON, np.array([[[float(c) for c in v] for v in verts]]), 3)[0]
    assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_symmetry_rowsums_and_total_mass(q):
    v = random_simplices(3, 16)
    vol = np.abs(np.einsum("ei,ei->e", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6
    M = element.element_tensors(MASS, v, q)
    A = element.element_tensors(POISSON, v, q)
    assert np.allclose(M, np.swapaxes(M, 1, 2), rtol=0, atol=1e-15 * np.abs(M).max())
    assert np.allclose(A, np.swapaxes(A, 1, 2), rtol=0, atol=1e-13 * np.abs(A).max())
    assert np.allclose(M.sum(axis=(1, 2)), vol, rtol=1e-13)
    assert np.abs(A.sum(axis=2)).max() < 1e-12 * np.abs(A).max()


def _interpolate(vfun, verts, d, q):
    """Nodal values of a function at the lattice nodes of each cell [E, n_s, ...]."""
    lam = np.array(basis.lattice(d, q), float) / q
    x = np.einsum("kj,ejx->ekx", lam, verts)
    return vfun(x)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_elasticity_rigid_modes_and_linear_fields(q):
    d = 3
    v = random_simplices(d, 8)
    A = element.element_tensors(ELASTICITY, v, q, mu=1.0, lmbda=1.25)
    ns = n_local(d, q)
    vol = np.abs(np.einsum("ei,ei->e", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6
    rng = np.random.default_rng(7)
    W = rng.standard_normal((3, 3)); W = W - W.T
    B = rng.standard_normal((3, 3))
    for mat, energy in [(W, 0.0), (B, None)]:
        u = _interpolate(lambda x: np.einsum("ab,ekb->eka", mat, x) + 0.3, v, d, q)  # [E, ns, 3]
        uvec = np.concatenate([u[:, :, c] for c in range(d)], axis=1)  # component blocked
        e_ = np.einsum("ei,eij,ej->e", uvec, A, uvec)
        S = 0.5 * (mat + mat.T)
        expect = vol * (2 * np.sum(S * S) + 1.25 * np.trace(mat) ** 2)
        if energy == 0.0:
            assert np.abs(np.einsum("eij,ej->ei", A, uvec)).max() < 1e-11 * np.abs(A).max()
        assert np.allclose(e_, expect, rtol=1e-11)


def test_convection_invariants():
    d, q = 3, 2
    v = random_simplices(d, 8)
    rng = np.random.default_rng(3)
    w1 = rng.standard_normal((8, 30)); w2 = rng.standard_normal((8, 30))
    A1 = element.element_tensors(NS_CONVECTION, v, q, coeffs=w1)
    A2 = element.element_tensors(NS_CONVECTION, v, q, coeffs=w2)
    A12 = element.element_tensors(NS_CONVECTION, v, q, coeffs=w1 + 2 * w2)
    assert np.allclose(A12, A1 + 2 * A2, rtol=0, atol=1e-12 * np.abs(A12).max())
    for c in range(d):  # constant vector fields are annihilated (grad const = 0)
        ones = np.zeros(30); ones[c * 10:(c + 1) * 10] = 1
        assert np.abs(A1 @ ones).max() < 1e-12 * np.abs(A1).max()
    # w = e_x, vector P1: A[(c,i),(c,j)] = int lambda_i d_x lambda_j = |K| d_x lambda_j / 4
    wx = np.zeros((8, 12)); wx[:, 0:4] = 1
    A = element.element_tensors(NS_CONVECTION, v, 1, coeffs=wx)
    gl, vol = element.barycentric_geometry(v)
    for c in range(3):
        blk = A[:, c * 4:(c + 1) * 4, c * 4:(c + 1) * 4]
        assert np.allclose(blk, (vol[:, None] * gl[:, :, 0] / 4)[:, None, :].repeat(4, 1), rtol=1e-12)
    off = A.copy()
    for c in range(3):
        off[:, c * 4:(c + 1) * 4, c * 4:(c + 1) * 4] = 0
    assert np.abs(off).max() == 0


@pytest.mark.parametrize("form,q", [(MASS, 4), (POISSON, 4), (ELASTICITY, 3), (NS_CONVECTION, 2)])
def test_brute_force_more_points_changes_nothing(form, q):
    v = random_simplices(3, 4)
    c = np.random.default_rng(1).standard_normal((4, 30)) if form == NS_CONVECTION else None
    A = element.element_tensors(form, v, q, coeffs=c)
    B = element.element_tensors(form, v, q, coeffs=c, extra_points=2)
    assert np.abs(A - B).max() <= 1e-14 * np.abs(A).max() * q


def test_negative_orientation_uses_absolute_determinant():
    v = random_simplices(3, 6)
    vf = v[:, [0, 2, 1, 3]]  # swap two vertices: same cell, opposite orientation
    for form, q in [(MASS, 2), (POISSON, 3)]:
        A = element.element_tensors(form, v, q)
        B = element.element_tensors(form, vf, q)
        perm = [basis.lattice(3, q).index(tuple(k[[0, 2, 1, 3]])) for k in np.array(basis.lattice(3, q))]
        assert np.allclose(B, A[:, perm][:, :, perm], rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- linear form (source)
@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("t", range(len(RATIONAL_TETS)))
def test_source_vector_vs_exact_rational(q, t):
    verts = [tuple(Fraction(c) for c in v) for v in RATIONAL_TETS[t]]
    n = n_local(3, q)
    f = [Fraction((5 * i) % 9 - 4, 7) for i in range(n)]
    ref = np.array(X.load_vector(verts, q, f), dtype=float)
    vf = np.array([[float(c) for c in v] for v in verts])[None]
    b = element.element_tensors(element.SOURCE, vf, q, coeffs=np.array([[float(x) for x in f]]))[0]
    assert np.abs(b - ref).max() <= 1e-14 * np.abs(ref).max()


def test_source_vector_closed_forms():
    v = random_simplices(3, 10)
    vol = np.abs(np.einsum("ei,ei->e", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6
    b = element.element_tensors(element.SOURCE, v, 1, coeffs=np.ones((10, 4)))
    assert np.allclose(b, vol[:, None] / 4, rtol=1e-14)  # int lambda_i = |K| / (d+1)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((10, 20))
    b = element.element_tensors(element.SOURCE, v, 3, coeffs=f)
    M = element.element_tensors(MASS, v, 3)
    assert np.allclose(b, np.einsum("eij,ej->ei", M, f), rtol=1e-12, atol=1e-15)  # b = M f
