"""Host-side parts of the product library, no GPU needed: the library loads and
exports every entry point of include/ffc_gb300.h, argument checks reject bad
calls before any launch, the form compiler's reference tensors match exact
rational values, and the CSR pattern builder matches an independent pattern."""
import ctypes
import os
import re

import numpy as np
import pytest

import exact_forms as X

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1112_0402_gb300 import _capi
    from paper_1112_0402_gb300 import build as B

    B.build()
    return _capi.lib()


def test_library_exports_every_declared_symbol():
    L = _lib()
    header = open(os.path.join(ROOT, "include", "ffc_gb300.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ffc_\w+)\s*\(", header, re.M))
    assert len(declared) >= 11
    from paper_1112_0402_gb300 import _capi

    assert declared == set(_capi.SIGNATURES)
    for name in declared:
        assert getattr(L, name) is not None


def test_form_create_validates_arguments():
    import paper_1112_0402_gb300 as F

    for bad in [(9, 3, 1), (1, 4, 1), (1, 3, 0), (1, 3, 5)]:
        with pytest.raises(F.FFCError) as e:
            F.Form(*bad)
        assert e.value.code == -1
    with pytest.raises(F.FFCError) as e:
        F.Form(F.NS_CONVECTION, F.TETRAHEDRON, 3)
    assert e.value.code == -5
    f = F.Form(F.NS_CONVECTION, F.TETRAHEDRON, 2)
    assert (f.n_local, f.n_alpha, f.n_coeff) == (30, 90, 30)
    f = F.Form(F.ELASTICITY, F.TETRAHEDRON, 3)
    assert (f.n_local, f.n_alpha, f.n_coeff) == (60, 81, 0)


def test_device_calls_reject_null_pointers_without_a_gpu():
    L = _lib()
    import paper_1112_0402_gb300 as F

    f = F.Form(F.POISSON, F.TETRAHEDRON, 1)
    # null cells with n_elem > 0 -> FFC_EINVAL before touching the device
    assert L.ffc_tabulate(f.handle, 10, None, None, 5, None, None, 0, None) == -1
    assert L.ffc_assemble(f.handle, 10, None, None, 5, None, None, None, 3, 0, None) == -1
    assert L.ffc_tabulate(f.handle, -1, None, None, 5, None, None, 0, None) == -1
    assert L.ffc_tabulate(f.handle, 10, None, None, 5, None, None, 99, None) == -1
    assert L.ffc_tabulate(None, 10, None, None, 5, None, None, 0, None) == -1
    assert L.ffc_status_string(-5).decode().startswith("FFC_EUNSUPPORTED")


def _A0(kind, cell, q):
    import paper_1112_0402_gb300 as F

    return F.Form(kind, cell, q).reference_tensor()


@pytest.mark.parametrize("d,q", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_poisson_and_mass_reference_tensors_vs_exact(d, q):
    import paper_1112_0402_gb300 as F

    n = X.n_local if hasattr(X, "n_local") else None  # noqa: F841
    exact = np.array(X.reference_tensor_poisson(d, q), dtype=float)  # [i1][i2][a1][a2]
    nl = exact.shape[0]
    A0 = _A0(F.POISSON, d, q).reshape(nl, nl, d, d)
    assert np.abs(A0 - exact).max() <= 4e-15 * np.abs(exact).max()
    exact_m = np.array(X.reference_tensor_mass(d, q), dtype=float)
    A0m = _A0(F.MASS, d, q).reshape(nl, nl)
    assert np.abs(A0m - exact_m).max() <= 4e-15 * np.abs(exact_m).max()


def test_printed_p3_triangle_reference_tensor_entries():
    import paper_1112_0402_gb300 as F

    A0 = _A0(F.POISSON, 2, 3).reshape(10, 10, 2, 2)
    # printed generated code (Section 5.5): 0.425 for all four G entries of block[0],
    # 4.05 / 2.025 / 2.025 / 4.05 for block[99]; G is symmetric so the printed
    # G0_a_b naming fixes only sums over (a, b) <-> (b, a)
    assert np.allclose(A0[0, 0], 0.425, atol=1e-14)
    assert np.allclose(A0[9, 9], [[4.05, 2.025], [2.025, 4.05]], atol=1e-14)
    assert abs(A0[0, 1].sum() - (-0.175)) < 1e-14 and abs(A0[0, 1, :, 1]).max() < 1e-15
    assert abs(A0[0, 2].sum() - (-0.175)) < 1e-14 and abs(A0[0, 2, :, 0]).max() < 1e-15


def test_p4_tet_reference_tensors_invariants():
    import paper_1112_0402_gb300 as F

    A0 = _A0(F.POISSON, 3, 4).reshape(35, 35, 3, 3)
    assert np.abs(A0.sum(axis=1)).max() < 1e-13  # sum_i2 Psi_i2 = 1 -> derivative 0
    assert np.abs(A0 - A0.transpose(1, 0, 3, 2)).max() < 1e-15
    M = _A0(F.MASS, 3, 4)
    assert abs(M.sum() - 1 / 6) < 1e-15


@pytest.mark.parametrize("q", [1, 2])
def test_convection_reference_tensor_vs_exact(q):
    import paper_1112_0402_gb300 as F

    S = np.array(X.reference_tensor_convection(3, q), dtype=float)  # [s1][s2][st][a]
    ns = S.shape[0]
    A0 = _A0(F.NS_CONVECTION, 3, q).reshape(3, ns, 3, ns, 3, ns, 3)  # c1 s1 c2 s2 ct st a
    for c1 in range(3):
        for c2 in range(3):
            for ct in range(3):
                blk = A0[c1, :, c2, :, ct]
                if c1 == c2:
                    assert np.abs(blk - S).max() <= 4e-15 * np.abs(S).max()
                else:
                    assert np.abs(blk).max() == 0


@pytest.mark.parametrize("q", [1, 2])
def test_elasticity_reference_tensor_structure(q):
    import paper_1112_0402_gb300 as F

    P = np.array(X.reference_tensor_poisson(3, q), dtype=float)
    ns = P.shape[0]
    A0 = _A0(F.ELASTICITY, 3, q).reshape(3, ns, 3, ns, 3, 3, 3, 3)  # c1 s1 c2 s2 b1 b2 a1 a2
    for c1 in range(3):
        for c2 in range(3):
            for b1 in range(3):
                for b2 in range(3):
                    blk = A0[c1, :, c2, :, b1, b2]
                    if (c1, c2) == (b1, b2):
                        assert np.abs(blk - P).max() <= 4e-15 * np.abs(P).max()
                    else:
                        assert np.abs(blk).max() == 0


@pytest.mark.parametrize("d,n,q", [(2, 3, 1), (2, 2, 3), (3, 2, 2), (3, 1, 4)])
def test_csr_pattern_and_slots(d, n, q):
    import paper_1112_0402_gb300 as F
    from synthetic import mesh as M
    from synthetic import workloads as W

    m = M.unit_square_triangles(n, 0.1, 3) if d == 2 else M.unit_cube_tets(n, 0.1, 3)
    p = W.make_problem(m, W.POISSON, q)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    # independent pattern: every (row, col) pair sharing a cell, via numpy unique
    pairs = np.unique(np.stack([np.repeat(p.dofmap, p.n_local, axis=1).ravel(),
                                np.tile(p.dofmap, (1, p.n_local)).ravel()], axis=1), axis=0)
    ref_ptr = np.concatenate([[0], np.cumsum(np.bincount(pairs[:, 0], minlength=p.n_dof))])
    assert np.array_equal(row_ptr, ref_ptr)
    assert np.array_equal(col, pairs[:, 1].astype(np.int32))
    rows = np.repeat(p.dofmap, p.n_local, axis=1).reshape(slot.shape)
    cols = np.tile(p.dofmap, (1, p.n_local)).reshape(slot.shape)
    assert np.all(slot >= row_ptr[rows]) and np.all(slot < row_ptr[rows + 1])
    assert np.array_equal(col[slot], cols)


def test_csr_pattern_rejects_out_of_range_dofs():
    import paper_1112_0402_gb300 as F

    dm = np.array([[0, 1, 7]], dtype=np.int32)
    with pytest.raises(F.FFCError) as e:
        F.csr_pattern(dm, 5)
    assert e.value.code == -6


def test_algorithm_and_batch_arguments_are_validated_on_the_host():
    import ctypes

    import paper_1112_0402_gb300 as F
    from paper_1112_0402_gb300 import _capi

    L = _lib()
    f = F.Form(F.ELASTICITY, F.TETRAHEDRON, 2, algorithm=F.ALG_BLOCK)
    assert L.ffc_form_set_algorithm(f.handle, 7) == -1
    assert L.ffc_form_set_algorithm(None, 0) == -1
    items = (_capi.BatchItem * 1)()
    items[0].form = f.handle
    items[0].n_elem = 10  # null device pointers: rejected before any device work
    out = ctypes.c_void_p()
    assert L.ffc_batch_create(items, 1, 1, ctypes.byref(out)) == -1
    g = F.Form(F.POISSON, F.TETRAHEDRON, 4)  # a form the batched kernel does not carry
    items[0].form = g.handle
    assert L.ffc_batch_create(items, 1, 1, ctypes.byref(out)) == -5
    assert L.ffc_batch_create(None, 0, 1, ctypes.byref(out)) == -1


@pytest.mark.parametrize("d,q", [(2, 1), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_source_form_is_rank_one_with_the_mass_reference_tensor(d, q):
    import paper_1112_0402_gb300 as F

    f = F.Form(F.SOURCE, d, q)
    exact = np.array(X.reference_tensor_mass(d, q), dtype=float)
    n = exact.shape[0]
    assert (f.rank, f.n_local, f.n_alpha, f.n_coeff) == (1, n, n, n)
    A0 = f.reference_tensor()
    assert A0.shape == (n, n)  # A0[i][t] = int Psi_i Psi_t
    assert np.abs(A0 - exact).max() <= 4e-15 * np.abs(exact).max()
    assert F.Form(F.MASS, d, q).rank == 2
    with pytest.raises(F.FFCError):
        F.Form(5, d, q)


def test_scatter_add_arguments_are_validated_on_the_host():
    L = _lib()
    # bad precision, empty entries, negative sizes, null pointers: rejected before any launch
    assert L.ffc_scatter_add(10, 4, None, 2, None, None, 5, None) == -1
    assert L.ffc_scatter_add(10, 0, None, 0, None, None, 5, None) == -1
    assert L.ffc_scatter_add(-1, 4, None, 0, None, None, 5, None) == -1
    assert L.ffc_scatter_add(10, 4, None, 0, None, None, 5, None) == -1
    assert L.ffc_scatter_add(10, 4, None, 0, None, None, 2**31, None) == -1
    assert L.ffc_scatter_add(0, 4, None, 0, None, None, 5, None) == 0  # nothing to do


def test_row_plan_and_row_assembly_arguments_are_validated_on_the_host():
    import ctypes

    import paper_1112_0402_gb300 as F

    L = _lib()
    out = ctypes.c_void_p()
    buf = np.zeros(64, dtype=np.int64)  # stands in for device pointers: never dereferenced
    fake = ctypes.c_void_p(buf.ctypes.data)
    assert L.ffc_row_plan_create(10, 4, None, 5, fake, fake, 8, None, ctypes.byref(out)) == -1  # no dofmap
    assert L.ffc_row_plan_create(10, 4, fake, 5, None, fake, 8, None, ctypes.byref(out)) == -1  # no row_ptr
    assert L.ffc_row_plan_create(10, 4, fake, 0, fake, fake, 8, None, ctypes.byref(out)) == -1  # no rows
    assert L.ffc_row_plan_create(10, 0, fake, 5, fake, fake, 8, None, ctypes.byref(out)) == -1  # no local dofs
    assert L.ffc_row_plan_create(10, 4, fake, 5, fake, fake, 8, None, None) == -1               # no output
    assert L.ffc_row_plan_create(2**29, 4, fake, 5, fake, fake, 8, None, ctypes.byref(out)) == -1  # E*n >= 2^31
    assert L.ffc_row_plan_info(None, None, None, None, None) == -1
    L.ffc_row_plan_destroy(None)
    f = F.Form(F.POISSON, F.TETRAHEDRON, 2)
    assert L.ffc_assemble_rows(f.handle, None, fake, fake, 5, fake, 1, None) == -1  # no plan
    assert L.ffc_assemble_rows(None, fake, fake, fake, 5, fake, 1, None) == -1      # no form
    assert L.ffc_assemble_rows(f.handle, fake, fake, fake, 5, fake, 2, None) == -1  # tensor-core precision


def test_bounded_wait_probe_limit_is_validated_on_the_host():
    L = _lib()
    assert L.ffc_diag_bounded_wait(2**20 + 1, None) == -1


def test_assemble_pair_arguments_are_validated_on_the_host():
    import paper_1112_0402_gb300 as F

    L = _lib()
    m2, p1 = F.Form(F.MASS, F.TETRAHEDRON, 2), F.Form(F.POISSON, F.TETRAHEDRON, 1)
    ns = F.Form(F.NS_CONVECTION, F.TETRAHEDRON, 2)
    buf = np.zeros(4)
    x, y = buf[:2].ctypes.data, buf[2:].ctypes.data
    assert L.ffc_assemble_pair(None, m2.handle, 0, None, None, 0, None, x, y, 0, 1, None) == -1
    assert L.ffc_assemble_pair(m2.handle, p1.handle, 0, None, None, 0, None, x, y, 0, 1, None) == -1  # spaces
    assert L.ffc_assemble_pair(m2.handle, m2.handle, 0, None, None, 0, None, x, x, 0, 1, None) == -1  # one array
    assert L.ffc_assemble_pair(ns.handle, ns.handle, 0, None, None, 0, None, x, y, 0, 1, None) == -5  # coefficients
