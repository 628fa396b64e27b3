"""Host side of the quadrature representation (Section 3.4), no GPU needed: the rule the
library compiles equals the oracle's independently written collapsed Gauss-Jacobi rule,
the reference tensor with a point index A~0 equals the weighted basis products the
oracle tabulates at those points, on affine cells A~0 summed over the points is the
tensor representation's A0 (the same integrals), and bad arguments are refused."""
import numpy as np
import pytest

from oracle import basis
from oracle import curved as OC


def _F():
    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    return F


def _match(Xa, Xb):
    """Permutation p with Xa[p] == Xb (points in different orders)."""
    ka = np.lexsort(Xa.T[::-1])
    kb = np.lexsort(Xb.T[::-1])
    p = np.empty(len(Xa), dtype=int)
    p[kb] = ka
    return p


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("p", [0, 2, 5, 7])
def test_rule_equals_the_oracle_rule(d, p):
    F = _F()
    qf = F.QForm(F.MASS, F.TRIANGLE if d == 2 else F.TETRAHEDRON, 1, 2, p)
    X, w = qf.rule()
    Xo, wo = OC.collapsed_rule(d, p)
    assert X.shape == Xo.shape
    perm = _match(X, Xo)
    assert np.abs(X[perm] - Xo).max() < 1e-15
    assert np.abs(w[perm] - wo).max() < 1e-14 * wo.max()


@pytest.mark.parametrize("d,form,q,g", [(2, 1, 2, 2), (3, 1, 2, 2), (3, 0, 3, 2), (2, 0, 1, 1), (3, 1, 3, 1)])
def test_reference_tensor_with_a_point_index(d, form, q, g):
    F = _F()
    p = 2 * q + d * (g - 1)
    qf = F.QForm(form, F.TRIANGLE if d == 2 else F.TETRAHEDRON, q, g, p)
    At = qf.reference_tensor()  # [n*n][K], K index = k * n_g + pair
    X, w = qf.rule()
    n, nq = qf.n_local, qf.n_points
    ng = 1 if form == 0 else d * (d + 1) // 2
    assert At.shape == (n * n, nq * ng)
    lam = np.concatenate([(1.0 - X.sum(axis=1))[:, None], X], axis=1)
    phi = basis.values(d, q, lam)
    dphi = OC.reference_gradients(d, q, X)
    pairs = [(a, a) for a in range(d)] + ([(0, 1)] if d == 2 else [(0, 1), (0, 2), (1, 2)])
    A = At.reshape(n, n, nq, ng)
    for k in range(nq):
        if form == 0:
            ref = w[k] * np.outer(phi[k], phi[k])
            assert np.abs(A[:, :, k, 0] - ref).max() < 1e-15
        else:
            for gi, (a, b) in enumerate(pairs):
                v = np.outer(dphi[k, :, a], dphi[k, :, b])
                if a != b:
                    v = v + np.outer(dphi[k, :, b], dphi[k, :, a])
                assert np.abs(A[:, :, k, gi] - w[k] * v).max() < 1e-13


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_point_sums_are_the_tensor_representation(d, q):
    """Affine cells: G~ is the same at every point, so sum_k A~0[i][(k, pair)] must be
    A0's column for that pair (A0 from the tensor representation's compiler)."""
    F = _F()
    cell = F.TRIANGLE if d == 2 else F.TETRAHEDRON
    qf = F.QForm(F.POISSON, cell, q, 1, 2 * q)
    n, nq = qf.n_local, qf.n_points
    ng = d * (d + 1) // 2
    S = qf.reference_tensor().reshape(n * n, nq, ng).sum(axis=1)
    A0 = F.Form(F.POISSON, cell, q).reference_tensor()  # [n*n][d*d], alpha = a1*d + a2
    pairs = [(a, a) for a in range(d)] + ([(0, 1)] if d == 2 else [(0, 1), (0, 2), (1, 2)])
    for gi, (a, b) in enumerate(pairs):
        col = A0[:, a * d + b] + (A0[:, b * d + a] if a != b else 0.0)
        assert np.abs(S[:, gi] - col).max() <= 1e-13 * np.abs(A0).max()
    qm = F.QForm(F.MASS, cell, q, 1, 2 * q)
    Sm = qm.reference_tensor().sum(axis=1)
    assert np.abs(Sm - F.Form(F.MASS, cell, q).reference_tensor()[:, 0]).max() < 1e-15


def test_qform_validates_arguments():
    F = _F()
    for bad in [(2, 3, 1, 2, 4), (1, 4, 1, 2, 4), (1, 3, 5, 2, 4), (1, 3, 1, 3, 4), (1, 3, 1, 2, 21), (1, 3, 1, 0, 4)]:
        with pytest.raises(F.FFCError) as e:
            F.QForm(*bad)
        assert e.value.code == -1
    qf = F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2, 7)
    assert (qf.n_local, qf.n_geometry, qf.n_points, qf.k_contract) == (10, 10, 64, 384)
    from paper_1112_0402_gb300 import _capi

    L = _capi.lib()
    # null cells with n_elem > 0, a bad precision: refused before any device work
    assert L.ffc_tabulate_quadrature(qf.handle, 4, None, None, 10, None, 0, None) == -1
    assert L.ffc_tabulate_quadrature(qf.handle, 4, None, None, 10, None, 7, None) == -1
    assert L.ffc_assemble_quadrature(qf.handle, 4, None, None, 10, None, None, 5, 0, None) == -1
    assert L.ffc_tabulate_quadrature(qf.handle, 0, None, None, 0, None, 0, None) == 0


def test_tensor_core_precisions_are_checked_before_device_work():
    """The tensor-core precisions take element tensors of at most 512 entries (refused with
    FFC_EUNSUPPORTED above); bad pointers are refused before any device work."""
    F = _F()
    from paper_1112_0402_gb300 import _capi

    L = _capi.lib()
    p4 = F.QForm(F.POISSON, F.TETRAHEDRON, 4, 2)  # 35 x 35 = 1225 entries, more than four M tiles
    p2 = F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2)
    for prec in (F.TF32, F.TF32X3, F.BF16X3):
        assert L.ffc_tabulate_quadrature(p4.handle, 4, None, None, 10, None, prec, None) == -5
        assert L.ffc_tabulate_quadrature(p2.handle, 4, None, None, 10, None, prec, None) == -1  # null cells
        assert L.ffc_assemble_quadrature(p2.handle, 4, None, None, 10, None, None, 5, prec, None) == -1


def test_digit_split_fp64_is_checked_before_device_work():
    """FFC_FP64_OZAKI: ffc_tabulate_quadrature only, element tensors of at most 128 entries
    and contractions of at most 400 terms (FFC_EUNSUPPORTED beyond)."""
    F = _F()
    from paper_1112_0402_gb300 import _capi

    L = _capi.lib()
    assert F.FP64_OZAKI == 5 and F.PRECISIONS["fp64_ozaki"] == 5
    p2 = F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2)   # 100 entries, 64 x 6 = 384 terms
    assert L.ffc_tabulate_quadrature(p2.handle, 4, None, None, 10, None, F.FP64_OZAKI, None) == -1  # null cells
    assert L.ffc_tabulate_quadrature(F.QForm(F.POISSON, F.TETRAHEDRON, 3, 2).handle, 4, None, None, 10, None,
                                     F.FP64_OZAKI, None) == -5
    assert L.ffc_tabulate_quadrature(F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2, 9).handle, 4, None, None, 10, None,
                                     F.FP64_OZAKI, None) == -5
    assert L.ffc_assemble_quadrature(p2.handle, 4, None, None, 10, None, None, 5, F.FP64_OZAKI, None) == -1
    # the tensor representation's entry points refuse it
    f = F.Form(F.POISSON, F.TETRAHEDRON, 2)
    assert L.ffc_tabulate(f.handle, 4, None, None, 10, None, None, F.FP64_OZAKI, None) == -1


def test_assembly_pointers_are_checked_before_device_work():
    """ffc_assemble_quadrature refuses null or misaligned slot / CSR pointers and a
    non-positive nnz with FFC_EINVAL, for every precision, before touching the device
    (the cell and node pointers below are never dereferenced)."""
    F = _F()
    from paper_1112_0402_gb300 import _capi

    L = _capi.lib()
    qf = F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2)
    cells, nodes = 4096, 8192  # aligned stand-ins, never read: the checks fail first
    for prec in (F.FP64, F.FP32, F.TF32X3, F.FP64_OZAKI):
        assert L.ffc_assemble_quadrature(qf.handle, 4, cells, nodes, 10, None, 16384, 5, prec, None) == -1
        assert L.ffc_assemble_quadrature(qf.handle, 4, cells, nodes, 10, 4098, 16384, 5, prec, None) == -1
        assert L.ffc_assemble_quadrature(qf.handle, 4, cells, nodes, 10, 4096, 16388, 5, prec, None) == -1
        assert L.ffc_assemble_quadrature(qf.handle, 4, cells, nodes, 10, 4096, 16384, 0, prec, None) == -1
