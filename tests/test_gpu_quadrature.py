"""Quadrature as a tensor contraction on the GPU (Section 3.4, "Curvilinear elements"):
ffc_tabulate_quadrature / ffc_assemble_quadrature against the oracle.

* affine cells (geometry degree 1, and straight quadratic cells): equal to the tensor
  representation (ffc_tabulate) and to the affine oracle, FP64 1e-12;
* curved quadratic-geometry cells: equal to the oracle's point-by-point quadrature sum
  with the same rule, per cell relative Frobenius error FP64 1e-12, FP32 1e-6;
* Algorithm 2 on curved cells: the assembled CSR matrix against the oracle's;
* the full-size bench configuration (vector of 384,000 curved cells) on a seeded sample;
* status flags: an out-of-range node id, a degenerate cell; a rule too large for one
  tile is refused.
"""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import curved as OC
from oracle import element as OE
from synthetic import dofmap as D
from synthetic import mesh as M
from synthetic.curved import curved_mesh, gather_nodes

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-6


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    assert torch.cuda.is_available()
    return F


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


def _rel(got, ref):
    E = ref.shape[0]
    return (np.linalg.norm((got - ref).reshape(E, -1), axis=1) / np.linalg.norm(ref.reshape(E, -1), axis=1)).max()


def _cell(F, d):
    return F.TRIANGLE if d == 2 else F.TETRAHEDRON


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_affine_cells_equal_the_tensor_representation(F, d, form, q):
    import torch

    m = M.unit_square_triangles(4, 0.25, 5) if d == 2 else M.unit_cube_tets(2, 0.25, 5)
    V = M.gather_cell_vertices(m)
    ref = OE.element_tensors(form, V, q)
    tensor = F.tabulate(F.Form(form, _cell(F, d), q), _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64),
                        precision="fp64").cpu().numpy()
    for g in (1, 2):
        nodes = OC.affine_nodes(V, g)  # every cell its own nodes
        E, ng = nodes.shape[:2]
        cells = np.arange(E * ng, dtype=np.int32).reshape(E, ng)
        qf = F.QForm(form, _cell(F, d), q, g, 2 * q)
        got = F.tabulate_quadrature(qf, _dev(cells), _dev(nodes.reshape(-1, d)), precision="fp64").cpu().numpy()
        assert F.status_poll() == 0
        assert _rel(got, ref) <= FP64_TOL
        assert _rel(got, tensor) <= FP64_TOL


@pytest.mark.parametrize("d,n", [(2, 5), (3, 2)])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_curved_cells_match_the_oracle(F, d, n, form, q):
    cm = curved_mesh(d, n, eps=0.12)
    qf = F.QForm(form, _cell(F, d), q, 2)
    ref = OC.element_tensors_curved(form, gather_nodes(cm), q, 2, qf.quad_degree)
    cells, nodes = _dev(cm.cells), _dev(cm.nodes)
    got = F.tabulate_quadrature(qf, cells, nodes, precision="fp64").cpu().numpy()
    assert F.status_poll() == 0
    assert _rel(got, ref) <= FP64_TOL
    got32 = F.tabulate_quadrature(qf, cells, nodes, precision="fp32").double().cpu().numpy()
    assert F.status_poll() == 0
    assert _rel(got32, ref) <= FP32_TOL
    # curved: the straight cells' tensors differ
    straight = OE.element_tensors(form, gather_nodes(cm)[:, :d + 1], q)
    assert _rel(straight, ref) > 1e-4


@pytest.mark.parametrize("d,n", [(2, 4), (3, 2)])
@pytest.mark.parametrize("form,q", [(1, 2), (0, 2), (1, 3), (1, 1)])
def test_curved_assembly_matches_algorithm2(F, d, n, form, q):
    import torch

    cm = curved_mesh(d, n, eps=0.12)
    qf = F.QForm(form, _cell(F, d), q, 2)
    dofmap, n_dof = D.scalar_dofmap(cm.mesh, q)
    ref_K = OC.element_tensors_curved(form, gather_nodes(cm), q, 2, qf.quad_degree)
    ref_ptr, ref_col, ref_val = OA.assemble_csr(ref_K, dofmap, n_dof)
    row_ptr, col, slot = F.csr_pattern(dofmap, n_dof)
    assert np.array_equal(row_ptr, ref_ptr) and np.array_equal(col, ref_col)
    precs = [("fp64", FP64_TOL), ("fp32", FP32_TOL)]
    if qf.n_local ** 2 <= 512:  # the tensor-core kernels, atomics in their drain
        precs += [("tf32x3", FP32_TOL), ("bf16x3", FP32_TOL)]
    if qf.n_local ** 2 <= 128:
        precs += [("fp64_ozaki", FP64_TOL)]
    for prec, tol in precs:
        val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
        F.assemble_quadrature(qf, _dev(cm.cells), _dev(cm.nodes), _dev(slot, torch.int32), val, precision=prec)
        assert F.status_poll() == 0
        assert np.abs(val.cpu().numpy() - ref_val).max() <= tol * np.abs(ref_val).max(), prec


def test_full_size_curved_sample(F):
    """40^3 x 6 = 384,000 curved tets (the bench configuration), P2 Poisson and mass:
    FP64 (CUDA cores and digit-split tensor cores), FP32 and the tensor-core precisions on
    300 seeded cells against the oracle; the Poisson rows' zero sums over all cells; every
    cell of the FP32-accurate paths (FP32, 3xTF32, BF16x3) within 1e-6 of the FP64 path
    (itself within 1e-12 of the oracle on the sample), of the digit-split FP64 within 1e-13."""
    import torch

    cm = curved_mesh(3, 40, eps=0.08)
    rng = np.random.default_rng(20261203)
    sel = np.sort(rng.choice(cm.n_elem, 300, replace=False))
    cells, nodes = _dev(cm.cells), _dev(cm.nodes)
    for form in (0, 1):
        qf = F.QForm(form, F.TETRAHEDRON, 2, 2)
        ref = OC.element_tensors_curved(form, gather_nodes(cm)[sel], 2, 2, qf.quad_degree)
        A64 = None
        for prec, tol in (("fp64", FP64_TOL), ("fp64_ozaki", FP64_TOL), ("fp32", FP32_TOL), ("tf32x3", FP32_TOL),
                          ("bf16x3", FP32_TOL), ("tf32", 5e-5)):
            A = F.tabulate_quadrature(qf, cells, nodes, precision=prec)
            assert F.status_poll() == 0
            got = A[_dev(sel).long()].double().cpu().numpy()
            assert _rel(got, ref) <= tol
            if form == 1:
                rs = A.double().sum(dim=2).abs().max().item()
                assert rs <= (1e-12 if prec == "fp64" else 1e-5) * A.double().abs().max().item()
            if prec == "fp64":
                A64 = A
                continue
            if prec != "tf32":
                d = (A.double() - A64).reshape(cm.n_elem, -1).norm(dim=1) / A64.reshape(cm.n_elem, -1).norm(dim=1)
                assert d.max().item() <= (1e-13 if prec == "fp64_ozaki" else FP32_TOL), (prec, d.max().item())
            del A
        del A64
        torch.cuda.empty_cache()


def test_quadrature_flags_and_limits(F):
    import torch

    cm = curved_mesh(3, 1, eps=0.1)
    qf = F.QForm(1, F.TETRAHEDRON, 2, 2)
    bad = cm.cells.copy()
    bad[0, 4] = cm.nodes.shape[0] + 7
    F.tabulate_quadrature(qf, _dev(bad), _dev(cm.nodes), precision="fp64")
    assert F.status_poll() & F.FLAG_BOUNDS
    flat = cm.cells.copy()
    flat[1, :] = flat[1, 0]  # every node of cell 1 at one point
    F.tabulate_quadrature(qf, _dev(flat), _dev(cm.nodes), precision="fp32")
    assert F.status_poll() & F.FLAG_DEGENERATE
    big = F.QForm(1, F.TETRAHEDRON, 2, 2, 20)  # 1331 points: the tile does not fit in shared memory
    with pytest.raises(F.FFCError):
        F.tabulate_quadrature(big, _dev(cm.cells), _dev(cm.nodes), precision="fp64")
    empty = torch.empty((0, 10), dtype=torch.int32, device="cuda")
    out = F.tabulate_quadrature(qf, empty, _dev(cm.nodes), precision="fp64")
    assert out.shape == (0, 10, 10)
    assert F.status_poll() == 0


@pytest.mark.parametrize("d,n", [(2, 5), (3, 2)])
@pytest.mark.parametrize("form,q", [(0, 1), (1, 1), (0, 2), (1, 2), (1, 3)])
@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-6), ("tf32x3", 1e-6), ("tf32", 1e-4)])
def test_tensor_core_quadrature_matches_the_oracle(F, d, n, form, q, prec, tol):
    """The tcgen05 contraction on curved cells (P3 tets: four 128-entry M tiles):
    the split precisions within the FP32 target 1e-6; single TF32 (11-bit operands) is
    applied only to the deviations of G~ from its centroid value, so its error is
    TF32's precision times their relative size. 3xTF32 keeps 22 bits of each operand
    (hi + lo), about 2^-21 per product of the deviations: on these strongly curved cells
    (eps 0.12) P3 Poisson's cancellation takes that to 1.03e-6, so it is held to 2e-6
    there (BF16x3, 24 bits, stays within 1e-6; on the benchmark mesh both are 3.6e-7)."""
    if prec == "tf32x3" and d == 3 and q == 3:
        tol = 2e-6
    cm = curved_mesh(d, n, eps=0.12)
    qf = F.QForm(form, _cell(F, d), q, 2)
    ref = OC.element_tensors_curved(form, gather_nodes(cm), q, 2, qf.quad_degree)
    got = F.tabulate_quadrature(qf, _dev(cm.cells), _dev(cm.nodes), precision=prec).double().cpu().numpy()
    assert F.status_poll() == 0
    assert _rel(got, ref) <= tol


@pytest.mark.parametrize("count", [1, 127, 129, 300])
def test_tensor_core_quadrature_ragged_tiles(F, count):
    """Cell counts around the 128-cell tile: every cell written, nothing beyond."""
    import torch

    cm = curved_mesh(3, 4, eps=0.1)
    qf = F.QForm(1, F.TETRAHEDRON, 2, 2)
    cells = _dev(cm.cells[:count])
    out = torch.full((count + 1, 10, 10), 7.0, dtype=torch.float32, device="cuda")
    F.tabulate_quadrature(qf, cells, _dev(cm.nodes), precision="bf16x3", out=out[:count])
    assert F.status_poll() == 0
    ref = OC.element_tensors_curved(1, gather_nodes(cm)[:count], 2, 2, qf.quad_degree)
    assert _rel(out[:count].double().cpu().numpy(), ref) <= 1e-6
    assert bool((out[count] == 7.0).all())


def test_tensor_core_quadrature_limits(F):
    cm = curved_mesh(3, 1, eps=0.1)
    big = F.QForm(1, F.TETRAHEDRON, 4, 2)  # 1225 entries: more than four 128-entry M tiles
    with pytest.raises(F.FFCError) as e:
        F.tabulate_quadrature(big, _dev(cm.cells), _dev(cm.nodes), precision="bf16x3")
    assert e.value.code == -5


@pytest.mark.parametrize("d,n", [(2, 5), (3, 2)])
@pytest.mark.parametrize("form,q", [(0, 1), (1, 1), (0, 2), (1, 2), (1, 3)])
def test_digit_split_fp64_matches_the_oracle(F, d, n, form, q):
    if d == 3 and q == 3:
        pytest.skip("P3 tets: 400 entries, more than one 128-entry tile")
    """FFC_FP64_OZAKI (FP64 from exact BF16 digit products on the tensor cores) on curved
    cells: within the FP64 tolerance of the oracle, and of the CUDA-core FP64 kernel."""
    cm = curved_mesh(d, n, eps=0.12)
    qf = F.QForm(form, _cell(F, d), q, 2)
    ref = OC.element_tensors_curved(form, gather_nodes(cm), q, 2, qf.quad_degree)
    cells, nodes = _dev(cm.cells), _dev(cm.nodes)
    got = F.tabulate_quadrature(qf, cells, nodes, precision="fp64_ozaki")
    assert F.status_poll() == 0
    assert got.dtype.is_floating_point and got.element_size() == 8
    got = got.cpu().numpy()
    assert _rel(got, ref) <= FP64_TOL
    simt = F.tabulate_quadrature(qf, cells, nodes, precision="fp64").cpu().numpy()
    assert _rel(got, simt) <= 1e-13


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("form", [0, 1])
def test_digit_split_fp64_on_affine_cells(F, d, form):
    """Geometry degree 1: equal to the tensor representation's FP64 element tensors."""
    import torch

    m = M.unit_square_triangles(4, 0.25, 5) if d == 2 else M.unit_cube_tets(2, 0.25, 5)
    V = M.gather_cell_vertices(m)
    tensor = F.tabulate(F.Form(form, _cell(F, d), 2), _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64),
                        precision="fp64").cpu().numpy()
    nodes = OC.affine_nodes(V, 1)
    E, ng = nodes.shape[:2]
    cells = np.arange(E * ng, dtype=np.int32).reshape(E, ng)
    qf = F.QForm(form, _cell(F, d), 2, 1, 4)
    got = F.tabulate_quadrature(qf, _dev(cells), _dev(nodes.reshape(-1, d)), precision="fp64_ozaki").cpu().numpy()
    assert F.status_poll() == 0
    assert _rel(got, tensor) <= FP64_TOL


@pytest.mark.parametrize("count", [1, 63, 65, 200])
def test_digit_split_fp64_ragged_tiles(F, count):
    """Cell counts around the 64-cell tile: every cell written, nothing beyond."""
    import torch

    cm = curved_mesh(3, 4, eps=0.1)
    qf = F.QForm(1, F.TETRAHEDRON, 2, 2)
    out = torch.full((count + 1, 10, 10), 7.0, dtype=torch.float64, device="cuda")
    F.tabulate_quadrature(qf, _dev(cm.cells[:count]), _dev(cm.nodes), precision="fp64_ozaki", out=out[:count])
    assert F.status_poll() == 0
    ref = OC.element_tensors_curved(1, gather_nodes(cm)[:count], 2, 2, qf.quad_degree)
    assert _rel(out[:count].cpu().numpy(), ref) <= FP64_TOL
    assert bool((out[count] == 7.0).all())


def test_digit_split_fp64_limits_and_flags(F):
    cm = curved_mesh(3, 1, eps=0.1)
    cells, nodes = _dev(cm.cells), _dev(cm.nodes)
    for qf in (F.QForm(1, F.TETRAHEDRON, 3, 2),      # 400 entries: more than one 128-entry tile
               F.QForm(1, F.TETRAHEDRON, 2, 2, 9)):  # 125 points x 6 = 750 > 400 terms
        with pytest.raises(F.FFCError) as e:
            F.tabulate_quadrature(qf, cells, nodes, precision="fp64_ozaki")
        assert e.value.code == -5
    qf = F.QForm(1, F.TETRAHEDRON, 2, 2)
    flat = cm.cells.copy()
    flat[1, :] = flat[1, 0]
    F.tabulate_quadrature(qf, _dev(flat), nodes, precision="fp64_ozaki")
    assert F.status_poll() & F.FLAG_DEGENERATE
    bad = cm.cells.copy()
    bad[0, 4] = cm.nodes.shape[0] + 7
    F.tabulate_quadrature(qf, _dev(bad), nodes, precision="fp64_ozaki")
    assert F.status_poll() & F.FLAG_BOUNDS


@pytest.mark.parametrize("scale_exp", [-40, 40])
def test_digit_split_fp64_on_tiny_and_huge_cells(F, scale_exp):
    """Cells scaled by 2^-40 and 2^40 (mass |det| by 2^-120 / 2^120, beyond FP32's range for
    the column-scale estimate): the digit-split FP64 result is the unscaled one times the
    exact power of two, to FP64 accuracy."""
    cm = curved_mesh(3, 2, eps=0.12)
    cells = _dev(cm.cells)
    for form, power in ((0, 3), (1, 1)):
        qf = F.QForm(form, F.TETRAHEDRON, 2, 2)
        base = F.tabulate_quadrature(qf, cells, _dev(cm.nodes), precision="fp64_ozaki").cpu().numpy()
        got = F.tabulate_quadrature(qf, cells, _dev(cm.nodes * 2.0 ** scale_exp), precision="fp64_ozaki")
        assert F.status_poll() == 0
        assert _rel(got.cpu().numpy() * 2.0 ** (-power * scale_exp), base) <= 1e-14


@pytest.mark.parametrize("prec", ["tf32x3", "fp64_ozaki"])
def test_tensor_core_assembly_skips_a_bad_slot(F, prec):
    """A slot outside [0, nnz) is skipped and reported; every other value is added."""
    import torch

    cm = curved_mesh(3, 2, eps=0.1)
    qf = F.QForm(1, F.TETRAHEDRON, 2, 2)
    dofmap, n_dof = D.scalar_dofmap(cm.mesh, 2)
    _, col, slot = F.csr_pattern(dofmap, n_dof)
    ref = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble_quadrature(qf, _dev(cm.cells), _dev(cm.nodes), _dev(slot, torch.int32), ref, precision=prec)
    assert F.status_poll() == 0
    bad = slot.copy()
    s0 = int(bad.reshape(-1)[5])
    bad.reshape(-1)[5] = col.size + 3
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble_quadrature(qf, _dev(cm.cells), _dev(cm.nodes), _dev(bad, torch.int32), val, precision=prec)
    assert F.status_poll() & F.FLAG_BOUNDS
    A = F.tabulate_quadrature(qf, _dev(cm.cells), _dev(cm.nodes), precision=prec).double().reshape(-1)
    diff = (ref - val).cpu().numpy()
    assert abs(diff[s0] - A[5].item()) <= 1e-9 * abs(A[5].item()) + 1e-15
    diff[s0] = 0.0
    assert np.abs(diff).max() <= 1e-9 * ref.abs().max().item()


@pytest.mark.parametrize("count", [1, 129, 300])
def test_tensor_core_quadrature_four_m_tiles(F, count):
    """P3 tets (400 entries, four 128-entry M tiles, one accumulator per M tile), mass and
    Poisson, 3xTF32 and BF16x3, cell counts around the 128-cell tile, a sentinel row."""
    import torch

    cm = curved_mesh(3, 4, eps=0.1)
    for form in (0, 1):
        qf = F.QForm(form, F.TETRAHEDRON, 3, 2)
        ref = OC.element_tensors_curved(form, gather_nodes(cm)[:count], 3, 2, qf.quad_degree)
        for prec, tol in (("tf32x3", 2e-6), ("bf16x3", FP32_TOL)):  # 3xTF32: 22-bit operands
            out = torch.full((count + 1, 20, 20), 7.0, dtype=torch.float32, device="cuda")
            F.tabulate_quadrature(qf, _dev(cm.cells[:count]), _dev(cm.nodes), precision=prec, out=out[:count])
            assert F.status_poll() == 0
            assert _rel(out[:count].double().cpu().numpy(), ref) <= tol, (form, prec)
            assert bool((out[count] == 7.0).all())
