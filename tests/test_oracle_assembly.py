"""Pins of the oracle's assembly (Algorithm 2) and shape derivative: the dict loop,
global closed forms on the unit square / cube, and finite differences."""
import numpy as np
import pytest

from oracle import assemble, element, shape
from oracle.element import ELASTICITY, MASS, NS_CONVECTION, POISSON, SOURCE
from synthetic import mesh as M
from synthetic import workloads as W


def _problem(d, n, form, q, jitter=0.15, seed=9):
    m = M.unit_square_triangles(n, jitter, seed) if d == 2 else M.unit_cube_tets(n, jitter, seed)
    return W.make_problem(m, form, q, seed=seed)


def _tensors(p):
    return element.element_tensors(p.form, M.gather_cell_vertices(p.mesh), p.degree, coeffs=p.coeffs)


@pytest.mark.parametrize("d,n,form,q", [(2, 3, POISSON, 1), (3, 1, MASS, 2), (3, 1, ELASTICITY, 1),
                                        (3, 1, NS_CONVECTION, 2)])
def test_sorted_assembly_equals_the_plain_loop(d, n, form, q):
    p = _problem(d, n, form, q)
    A_K = _tensors(p)
    rp, col, val = assemble.assemble_csr(A_K, p.dofmap, p.n_dof)
    ref = assemble.assemble_loop(A_K, p.dofmap)
    assert len(ref) == col.size
    for r in range(p.n_dof):
        for k in range(rp[r], rp[r + 1]):
            assert abs(ref[(r, int(col[k]))] - val[k]) <= 1e-14 * max(1.0, abs(val).max())
    assert np.all(np.diff(col[rp[0]:rp[1]]) > 0)
    rp2, col2 = assemble.csr_pattern(p.dofmap, p.n_dof)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def _nodal(p, f):
    """Global nodal vector of f at the dof points (lattice points of the jittered cells)."""
    from oracle import basis
    d, q = p.mesh.dim, p.degree
    lam = np.array(basis.lattice(d, q), float) / q
    x = np.einsum("kj,ejx->ekx", lam, M.gather_cell_vertices(p.mesh))
    out = np.zeros(p.n_dof)
    out[p.dofmap[:, :lam.shape[0]]] = f(x)
    return out


@pytest.mark.parametrize("d,n,q", [(2, 4, 1), (2, 3, 2), (3, 2, 1), (3, 2, 2), (3, 1, 3), (3, 1, 4)])
def test_global_mass_and_stiffness_reproduce_polynomial_integrals(d, n, q):
    pm = _problem(d, n, MASS, q)
    pa = _problem(d, n, POISSON, q)
    rp, col, Mv = assemble.assemble_csr(_tensors(pm), pm.dofmap, pm.n_dof)
    rpa, cola, Av = assemble.assemble_csr(_tensors(pa), pa.dofmap, pa.n_dof)
    assert abs(Mv.sum() - 1.0) < 1e-13  # partition of unity: sum of all entries = |Omega|
    assert np.abs(assemble.csr_matvec(rpa, cola, Av, np.ones(pa.n_dof))).max() < 1e-12
    if q == 1:
        a = np.array([0.3, -1.1, 0.7][:d])
        u = _nodal(pm, lambda x: x @ a + 0.5)
        Mu = assemble.csr_matvec(rp, col, Mv, u)
        exact_l2 = (0.5**2 + 0.5 * a.sum() + sum(a[i] * a[j] * (1 / 3 if i == j else 1 / 4)
                                                  for i in range(d) for j in range(d)))
        assert abs(u @ Mu - exact_l2) < 1e-13
        Au = assemble.csr_matvec(rpa, cola, Av, u)
        assert abs(u @ Au - a @ a) < 1e-12
    else:
        u = _nodal(pm, lambda x: x[..., 0] ** 2)
        assert abs(u @ assemble.csr_matvec(rp, col, Mv, u) - 1 / 5) < 1e-13
        assert abs(u @ assemble.csr_matvec(rpa, cola, Av, u) - 4 / 3) < 1e-12


def test_global_elasticity_energy_of_a_linear_field():
    p = _problem(3, 2, ELASTICITY, 2)
    rp, col, val = assemble.assemble_csr(_tensors(p), p.dofmap, p.n_dof)
    B = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.6], [0.25, 0.05, -0.1]])
    u = np.zeros(p.n_dof)
    sc = W.make_problem(p.mesh, POISSON, 2)
    for c in range(3):
        uc = _nodal(sc, lambda x: x @ B[c])
        u[c::3] = uc
    energy = u @ assemble.csr_matvec(rp, col, val, u)
    S = 0.5 * (B + B.T)
    assert abs(energy - (2 * np.sum(S * S) + 1.25 * np.trace(B) ** 2)) < 1e-12


def test_global_convection_skew_part_is_a_boundary_term():
    # for constant w = e_x: 1^T A 1 = int d_x (1) = 0 and A + A^T = boundary flux term,
    # which vanishes for functions that are zero on the boundary
    p = _problem(3, 2, NS_CONVECTION, 2)
    p.coeffs = np.zeros_like(p.coeffs)
    p.coeffs[:, :10] = 1.0
    rp, col, val = assemble.assemble_csr(_tensors(p), p.dofmap, p.n_dof)
    sc = W.make_problem(p.mesh, POISSON, 2)
    bubble = _nodal(sc, lambda x: np.prod(x * (1 - x), axis=-1))
    g = _nodal(sc, lambda x: np.sin(x[..., 0]) + x[..., 1] ** 2)
    u = np.zeros(p.n_dof); u[0::3] = bubble
    v = np.zeros(p.n_dof); v[0::3] = bubble * 0.7
    Au = assemble.csr_matvec(rp, col, val, u)
    Av = assemble.csr_matvec(rp, col, val, v)
    assert abs(v @ Au + u @ Av) < 1e-13  # skew on functions vanishing on the boundary
    one = np.zeros(p.n_dof); one[1::3] = 1.0
    assert np.abs(assemble.csr_matvec(rp, col, val, one)).max() < 1e-12
    assert g.shape == bubble.shape


@pytest.mark.parametrize("q", [1, 2])
def test_shape_gradient_matches_central_differences(q):
    p = _problem(3, 2, POISSON, q, jitter=0.15, seed=5)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(p.n_dof)
    v = rng.standard_normal(p.n_dof)
    x = p.mesh.vertices.copy()
    grad = shape.poisson_shape_gradient(x, p.mesh.cells, q, p.dofmap, u, v)
    h = 1e-6
    for k in rng.choice(x.shape[0], size=6, replace=False):
        for c in range(3):
            xp = x.copy(); xp[k, c] += h
            xm = x.copy(); xm[k, c] -= h
            fd = (shape.poisson_objective(xp, p.mesh.cells, q, p.dofmap, u, v)
                  - shape.poisson_objective(xm, p.mesh.cells, q, p.dofmap, u, v)) / (2 * h)
            assert abs(fd - grad[k, c]) < 1e-6 * max(1.0, abs(grad).max())
    # translation invariance: the gradient sums to zero over all vertices
    assert np.abs(grad.sum(axis=0)).max() < 1e-10 * np.abs(grad).max()


@pytest.mark.parametrize("d,n,q", [(2, 4, 1), (2, 3, 2), (3, 2, 1), (3, 2, 2), (3, 1, 3), (3, 1, 4)])
def test_global_load_vector_reproduces_polynomial_integrals(d, n, q):
    # b_i = int psi_i f; with f interpolated exactly (degree <= q), b . 1 = int f and
    # b . X = int x f for the nodal vector X of a linear x (q >= 1 reproduces it)
    p = _problem(d, n, SOURCE, q)
    for f, x_f in ((lambda x: 1.0 + 0 * x[..., 0], 1 / 2),
                   (lambda x: x[..., 0], 1 / 3)):
        p.coeffs = np.ascontiguousarray(_nodal(p, f)[p.dofmap])
        b = assemble.assemble_vector(_tensors(p), p.dofmap, p.n_dof)
        assert abs(b.sum() - (1.0 if x_f == 1 / 2 else 1 / 2)) < 1e-13
        X = _nodal(p, lambda x: x[..., 0])
        assert abs(b @ X - x_f) < 1e-13
    # loop form of Algorithm 2 for a vector
    ref = np.zeros(p.n_dof)
    bK = _tensors(p)
    for e in range(p.n_elem):
        for i in range(p.n_local):
            ref[p.dofmap[e, i]] += bK[e, i]
    assert np.array_equal(assemble.assemble_vector(bK, p.dofmap, p.n_dof), ref) or \
        np.abs(assemble.assemble_vector(bK, p.dofmap, p.n_dof) - ref).max() < 1e-15
