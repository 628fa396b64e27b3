"""Parity of the tcgen05 (tensor-core) contraction with the CPU oracle, tabulate and
fused assembly, ragged tails.

Tolerances (per-cell relative Frobenius error):
  bf16x3  1e-6   three BF16 parts per operand leave a residual below 2^-24 |x|, so the
                 six-product sum is as accurate as an FP32 contraction.
  tf32x3  3e-6   two TF32 parts leave a residual up to 2^-22 |x| per operand; the three
                 dropped product terms give up to 3 * 2^-22 = 7.2e-7 per product, which
                 cancellation inside A0 : G (random convection fields) amplifies ~4x.
  tf32    5e-3   one TF32 part: 2^-11 per operand."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

BF16X3_TOL = 1e-6
TF32X3_TOL = 3e-6
TF32_TOL = 5e-3


@pytest.fixture(scope="module")
def F():
    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    return F


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


TC_CASES = [(W.NS_CONVECTION, 2, 3), (W.ELASTICITY, 1, 3), (W.ELASTICITY, 2, 2), (W.ELASTICITY, 3, 2),
            (W.POISSON, 2, 3), (W.POISSON, 3, 3), (W.POISSON, 4, 2), (W.MASS, 3, 3), (W.MASS, 4, 2)]


@pytest.mark.parametrize("form,q,n", TC_CASES)
@pytest.mark.parametrize("prec,tol", [("bf16x3", BF16X3_TOL), ("tf32x3", TF32X3_TOL), ("tf32", TF32_TOL)])
def test_tc_tabulate_matches_oracle(F, form, q, n, prec, tol):
    import torch

    m = M.unit_cube_tets(n, 0.2, seed=23)
    p = W.make_problem(m, form, q, seed=23)
    ref = OE.element_tensors(form, M.gather_cell_vertices(m), q, coeffs=p.coeffs)
    fm = F.Form(form, F.TETRAHEDRON, q)
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    A = F.tabulate(fm, _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64), coeffs=coeffs, precision=prec)
    assert F.status_poll() == 0
    err = OE.frobenius_rel_error(A.double().cpu().numpy(), ref)
    assert err.max() <= tol, f"{prec} max rel err {err.max():.3e}"


@pytest.mark.parametrize("count", [1, 127, 129, 300])
def test_tc_ragged_tails(F, count):
    import torch

    m = M.unit_cube_tets(4, 0.2, seed=5)
    p = W.make_problem(m, W.NS_CONVECTION, 2, seed=5)
    ref = OE.element_tensors(W.NS_CONVECTION, M.gather_cell_vertices(m)[:count], 2, coeffs=p.coeffs[:count])
    fm = F.Form(W.NS_CONVECTION, F.TETRAHEDRON, 2)
    A = F.tabulate(fm, _dev(m.cells[:count], torch.int32), _dev(m.vertices, torch.float64),
                   coeffs=_dev(p.coeffs[:count], torch.float64), precision="bf16x3")
    assert F.status_poll() == 0
    assert OE.frobenius_rel_error(A.double().cpu().numpy(), ref).max() <= BF16X3_TOL


@pytest.mark.parametrize("form,q", [(W.NS_CONVECTION, 2), (W.ELASTICITY, 2), (W.POISSON, 3)])
def test_tc_assemble_matches_oracle(F, form, q):
    import torch

    m = M.unit_cube_tets(3, 0.2, seed=31)
    p = W.make_problem(m, form, q, seed=31)
    _, _, ref_val = OA.assemble_csr(OE.element_tensors(form, M.gather_cell_vertices(m), q, coeffs=p.coeffs),
                                    p.dofmap, p.n_dof)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    F.assemble(F.Form(form, F.TETRAHEDRON, q), _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64),
               _dev(slot, torch.int32), val, coeffs=coeffs, precision="bf16x3")
    assert F.status_poll() == 0
    got = val.cpu().numpy()
    assert np.linalg.norm(got - ref_val) <= BF16X3_TOL * np.linalg.norm(ref_val)


def test_tc_full_size_convection_sampled(F):
    """40^3 x 6 = 384,000 tets, vector P2 convection (the N-S workload), BF16x3:
    a seeded sample of 400 cells against the oracle."""
    import torch

    p = W.ns_vp2(40)
    m = p.mesh
    fm = F.Form(W.NS_CONVECTION, F.TETRAHEDRON, 2)
    A = F.tabulate(fm, _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64),
                   coeffs=_dev(p.coeffs, torch.float64), precision="bf16x3")
    assert F.status_poll() == 0
    idx = np.sort(np.random.default_rng(3).choice(m.n_elem, 400, replace=False))
    idx[-1] = m.n_elem - 1
    ref = OE.element_tensors(W.NS_CONVECTION, m.vertices[m.cells[idx]], 2, coeffs=p.coeffs[idx])
    got = A[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    assert OE.frobenius_rel_error(got, ref).max() <= BF16X3_TOL
