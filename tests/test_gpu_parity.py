"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element, on seeded meshes that span several tiles and a ragged tail; plus edge
cases (empty and single-cell inputs, degenerate cells, out-of-range slots) and
sampled checks at the full 48^3 x 6 tetrahedral workload size."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # per-element relative Frobenius error, FP64 contraction
FP32_TOL = 1e-6    # mixed-precision target


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    assert torch.cuda.is_available()
    return F


_PATTERNS = {}


def _pattern(F, p):
    key = (p.mesh.n, p.degree, p.n_dof)
    if key not in _PATTERNS:
        _PATTERNS.clear()
        _PATTERNS[key] = F.csr_pattern(p.dofmap, p.n_dof)
    return _PATTERNS[key]


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


def _case(d, n, form, q, seed=17, jitter=0.2):
    m = M.unit_square_triangles(n, jitter, seed) if d == 2 else M.unit_cube_tets(n, jitter, seed)
    return W.make_problem(m, form, q, seed=seed)


def _oracle(p):
    return OE.element_tensors(p.form, M.gather_cell_vertices(p.mesh), p.degree, coeffs=p.coeffs)


def _run_tabulate(F, p, precision, algorithm=0):
    import torch

    form = F.Form(p.form, p.mesh.dim, p.degree, algorithm=algorithm)
    cells = _dev(p.mesh.cells, torch.int32)
    verts = _dev(p.mesh.vertices, torch.float64)
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    A = F.tabulate(form, cells, verts, coeffs=coeffs, precision=precision)
    assert F.status_poll() == 0
    return A.double().cpu().numpy()


CASES = [(2, 7, W.POISSON, 1), (2, 5, W.POISSON, 3), (2, 5, W.MASS, 2), (2, 4, W.MASS, 4), (2, 4, W.POISSON, 4),
         (3, 3, W.MASS, 1), (3, 3, W.MASS, 2), (3, 3, W.MASS, 3), (3, 2, W.MASS, 4),
         (3, 3, W.POISSON, 1), (3, 3, W.POISSON, 2), (3, 3, W.POISSON, 3), (3, 2, W.POISSON, 4),
         (3, 3, W.NS_CONVECTION, 1), (3, 2, W.NS_CONVECTION, 2),
         (3, 3, W.ELASTICITY, 1), (3, 2, W.ELASTICITY, 2), (3, 2, W.ELASTICITY, 3)]


@pytest.mark.parametrize("d,n,form,q", CASES)
def test_tabulate_fp64_matches_oracle(F, d, n, form, q):
    p = _case(d, n, form, q)
    ref = _oracle(p)
    got = _run_tabulate(F, p, "fp64")
    err = OE.frobenius_rel_error(got, ref)
    assert err.max() <= FP64_TOL, f"max rel err {err.max():.3e}"


@pytest.mark.parametrize("d,n,form,q", CASES)
def test_tabulate_fp32_within_mixed_tolerance(F, d, n, form, q):
    p = _case(d, n, form, q)
    ref = _oracle(p)
    got = _run_tabulate(F, p, "fp32")
    err = OE.frobenius_rel_error(got, ref)
    assert err.max() <= FP32_TOL, f"max rel err {err.max():.3e}"


VECTOR_CASES = [c for c in CASES if c[2] in (W.NS_CONVECTION, W.ELASTICITY)]


@pytest.mark.parametrize("d,n,form,q", VECTOR_CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
@pytest.mark.parametrize("alg", ["dense", "block"])
def test_vector_forms_dense_and_block_algorithms(F, d, n, form, q, prec, tol, alg):
    """Both evaluations of the vector forms: the full reference tensor, and the
    Cartesian-product blocks (reduced reference tensor, reduced geometry)."""
    p = _case(d, n, form, q)
    got = _run_tabulate(F, p, prec, algorithm=F.ALG_DENSE if alg == "dense" else F.ALG_BLOCK)
    err = OE.frobenius_rel_error(got, _oracle(p))
    assert err.max() <= tol, f"{alg} {prec} max rel err {err.max():.3e}"


@pytest.mark.parametrize("form,q", [(W.NS_CONVECTION, 2), (W.ELASTICITY, 3)])
@pytest.mark.parametrize("alg", ["dense", "block"])
def test_vector_forms_assemble_both_algorithms(F, form, q, alg):
    import torch

    p = _case(3, 2, form, q)
    _, _, ref_val = OA.assemble_csr(_oracle(p), p.dofmap, p.n_dof)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    fm = F.Form(form, 3, q, algorithm=F.ALG_DENSE if alg == "dense" else F.ALG_BLOCK)
    F.assemble(fm, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64), _dev(slot, torch.int32),
               val, coeffs=coeffs, precision="fp64")
    assert F.status_poll() == 0
    got = val.cpu().numpy()
    assert np.linalg.norm(got - ref_val) <= FP64_TOL * np.linalg.norm(ref_val)


@pytest.mark.parametrize("d,n,form,q,prec", [(2, 6, W.POISSON, 1, "fp64"), (3, 3, W.MASS, 2, "fp64"),
                                               (3, 2, W.POISSON, 4, "fp64"), (3, 2, W.NS_CONVECTION, 2, "fp64"),
                                               (3, 2, W.ELASTICITY, 2, "fp64"), (3, 3, W.POISSON, 3, "fp32"),
                                               (3, 2, W.ELASTICITY, 3, "fp32")])
def test_assemble_matches_oracle_algorithm2(F, d, n, form, q, prec):
    import torch

    p = _case(d, n, form, q)
    ref_ptr, ref_col, ref_val = OA.assemble_csr(_oracle(p), p.dofmap, p.n_dof)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    assert np.array_equal(row_ptr, ref_ptr) and np.array_equal(col, ref_col)  # bit-exact structure
    form_ = F.Form(p.form, d, q)
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    F.assemble(form_, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64),
               _dev(slot, torch.int32), val, coeffs=coeffs, precision=prec)
    assert F.status_poll() == 0
    got = val.cpu().numpy()
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert np.linalg.norm(got - ref_val) <= tol * np.linalg.norm(ref_val)
    assert np.abs(got - ref_val).max() <= 10 * tol * np.abs(ref_val).max()


def test_empty_single_and_ragged_inputs(F):
    import torch

    p = _case(3, 3, W.POISSON, 2)
    form = F.Form(W.POISSON, 3, 2)
    verts = _dev(p.mesh.vertices, torch.float64)
    cells = _dev(p.mesh.cells, torch.int32)
    out = torch.zeros((0, 10, 10), dtype=torch.float64, device="cuda")
    F.tabulate(form, cells[:0], verts, out=out)
    ref = _oracle(p)
    for count in (1, 2, 31, 33, 65, 97, 161):
        sub = cells[:count].contiguous()
        A = F.tabulate(form, sub, verts).cpu().numpy()
        assert OE.frobenius_rel_error(A, ref[:count]).max() <= FP64_TOL
    assert F.status_poll() == 0


def test_degenerate_cell_sets_status_flag(F):
    import torch

    form = F.Form(W.POISSON, 3, 1)
    verts = _dev(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.5, 0.5, 0.0], [0, 0, 1]], float), torch.float64)
    cells = _dev(np.array([[0, 1, 2, 4], [0, 1, 2, 3]], np.int32), torch.int32)  # second is flat
    F.tabulate(form, cells[:1].contiguous(), verts)
    assert F.status_poll() == 0
    F.tabulate(form, cells, verts)
    assert F.status_poll() & F.FLAG_DEGENERATE
    assert F.status_poll() == 0  # poll clears


@pytest.mark.parametrize("form", [W.POISSON, W.MASS, W.SOURCE])
def test_degeneracy_threshold_of_a_sliver(F, form):
    """|det J| <= 1e-14 h_max^3 flags the cell: the sliver (0,0,0), (1,0,0), (0,1,0),
    (1/2, 1/2, eps) has det J = eps and h_max = sqrt(2), so the threshold is
    eps = 2.83e-14; both the full geometry (J^{-1}) and the determinant-only path."""
    import torch

    fm = F.Form(form, 3, 2)
    cells = _dev(np.array([[0, 1, 2, 3]], np.int32), torch.int32)
    coeffs = _dev(np.ones((1, 10)), torch.float64) if form == W.SOURCE else None
    for eps, flagged in ((1e-12, False), (4e-14, False), (2e-14, True), (1e-15, True)):
        verts = _dev(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.5, 0.5, eps]], float), torch.float64)
        F.tabulate(fm, cells, verts, coeffs=coeffs)
        assert bool(F.status_poll() & F.FLAG_DEGENERATE) == flagged, eps


@pytest.mark.parametrize("d,n,form,q,prec", [(3, 3, W.POISSON, 2, "fp64"), (3, 2, W.MASS, 4, "fp32"),
                                               (2, 5, W.POISSON, 3, "fp64"), (3, 2, W.ELASTICITY, 2, "fp32"),
                                               (3, 2, W.NS_CONVECTION, 2, "fp64")])
def test_scatter_add_of_tabulated_tensors_equals_fused_assembly(F, d, n, form, q, prec):
    """Algorithm 2's insertion on its own (tabulate, then scatter) gives the fused
    assembly's matrix and the oracle's."""
    import torch

    p = _case(d, n, form, q)
    row_ptr, col, slot = _pattern(F, p)
    fm = F.Form(p.form, d, q)
    cells, verts = _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64)
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    sl = _dev(slot, torch.int32)
    fused = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble(fm, cells, verts, sl, fused, coeffs=coeffs, precision=prec)
    A = F.tabulate(fm, cells, verts, coeffs=coeffs, precision=prec)
    split = torch.zeros_like(fused)
    F.scatter_add(A, sl, split)
    assert F.status_poll() == 0
    scale = fused.abs().max().item()
    assert (split - fused).abs().max().item() <= 1e-13 * scale
    ref = OA.assemble_csr(_oracle(p), p.dofmap, p.n_dof)[2]
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert np.linalg.norm(split.cpu().numpy() - ref) <= tol * np.linalg.norm(ref)


def test_scatter_add_edge_cases(F):
    import torch

    # ragged length (not a multiple of 4), an unaligned view, and an out-of-range slot
    vals = torch.arange(1, 12, dtype=torch.float32, device="cuda").reshape(11, 1)
    sl = torch.tensor([[0], [1], [2], [3], [4], [5], [6], [7], [8], [9], [2]], dtype=torch.int32, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    F.scatter_add(vals, sl, out)
    assert F.status_poll() == 0
    want = np.arange(1, 11, dtype=float)
    want[2] += 11
    assert np.array_equal(out.cpu().numpy(), want)
    out.zero_()
    F.scatter_add(vals[1:], sl[1:], out)  # views that start 4 bytes past a 16-byte boundary
    F.scatter_add(torch.ones((0, 3), dtype=torch.float64, device="cuda"),
                  torch.zeros((0, 3), dtype=torch.int32, device="cuda"), out)
    assert F.status_poll() == 0
    want = np.zeros(10)
    for v, k in zip(range(2, 12), [1, 2, 3, 4, 5, 6, 7, 8, 9, 2]):
        want[k] += v
    assert np.array_equal(out.cpu().numpy(), want)
    bad = sl.clone()
    bad[5, 0] = 10
    out.zero_()
    F.scatter_add(vals, bad, out)
    assert F.status_poll() == F.FLAG_BOUNDS
    assert out.sum().item() == pytest.approx(66.0 - 6.0)


def test_gathered_vertices_through_iota_cells(F):
    """Per-cell (gathered) vertex coordinates are accepted through cells[e] = (d+1)e + j:
    the same element tensors as the indexed form."""
    import torch

    p = _case(3, 3, W.POISSON, 3)
    fm = F.Form(W.POISSON, 3, 3)
    gathered = M.gather_cell_vertices(p.mesh).reshape(-1, 3)
    iota = np.arange(p.n_elem * 4, dtype=np.int32).reshape(p.n_elem, 4)
    a = F.tabulate(fm, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64))
    b = F.tabulate(fm, _dev(iota, torch.int32), _dev(gathered, torch.float64))
    assert F.status_poll() == 0
    assert torch.equal(a, b)


def test_out_of_range_slot_is_skipped_and_flagged(F):
    import torch

    p = _case(3, 2, W.MASS, 1)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    bad = slot.copy()
    bad[3, 1, 2] = col.size + 5
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble(F.Form(W.MASS, 3, 1), _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64),
               _dev(bad, torch.int32), val)
    assert F.status_poll() & F.FLAG_BOUNDS
    ref_ptr, ref_col, ref_val = OA.assemble_csr(_oracle(p), p.dofmap, p.n_dof)
    got = val.cpu().numpy()
    miss = slot[3, 1, 2]
    diff = np.abs(got - ref_val)
    diff[miss] = 0
    assert diff.max() <= 1e-13 * np.abs(ref_val).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("form,q", [(W.POISSON, 2), (W.MASS, 4), (W.POISSON, 4)])
def test_full_size_tet_workload_sampled(F, form, q, prec):
    """48^3 x 6 = 663,552 tets, the launch configuration of the benchmark; the oracle
    checks a seeded sample of 600 cells, and the whole assembled matrix is checked
    through properties that hold at any size."""
    import torch

    mesh = W.tet_scalar_mesh(48)
    p = W.make_problem(mesh, form, q)
    cells = _dev(mesh.cells, torch.int32)
    verts = _dev(mesh.vertices, torch.float64)
    fm = F.Form(form, 3, q)
    A = F.tabulate(fm, cells, verts, precision=prec)
    assert F.status_poll() == 0
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(mesh.n_elem, 600, replace=False))
    idx[-1] = mesh.n_elem - 1
    ref = OE.element_tensors(form, mesh.vertices[mesh.cells[idx]], q)
    err = OE.frobenius_rel_error(A[torch.as_tensor(idx, device="cuda")].double().cpu().numpy(), ref)
    assert err.max() <= (FP64_TOL if prec == "fp64" else FP32_TOL)
    del A
    row_ptr, col, slot = _pattern(F, p)
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble(fm, cells, verts, _dev(slot, torch.int32), val, precision=prec)
    assert F.status_poll() == 0
    tol = 1e-11 if prec == "fp64" else 1e-6
    if form == W.MASS:
        assert abs(val.sum().item() - 1.0) < tol  # total mass = |Omega|
    else:
        rows = torch.repeat_interleave(torch.arange(p.n_dof, device="cuda"), torch.as_tensor(np.diff(row_ptr),
                                                                                          device="cuda"))
        rs = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda").index_add_(0, rows, val)
        assert rs.abs().max().item() < tol * val.abs().max().item() * 10


@pytest.mark.parametrize("form,q", [(W.NS_CONVECTION, 1), (W.NS_CONVECTION, 2), (W.ELASTICITY, 1),
                                    (W.ELASTICITY, 2), (W.ELASTICITY, 3)])
def test_block_tabulate_ragged_counts(F, form, q):
    """The FP32 block kernels write A_K through shared-memory staging and bulk copies of a
    few cells at a time: every cell count (chunk and tile remainders) must come out
    complete and exact, with nothing written past the last cell."""
    import torch

    p = _case(3, 3, form, q)
    ref = _oracle(p)
    fm = F.Form(form, 3, q, algorithm=F.ALG_BLOCK)
    cells = _dev(p.mesh.cells, torch.int32)
    verts = _dev(p.mesh.vertices, torch.float64)
    coeffs = _dev(p.coeffs, torch.float64) if p.coeffs is not None else None
    n = p.n_local
    for count in (1, 2, 3, 4, 5, 63, 64, 65, 129, p.n_elem):
        out = torch.full((count + 1, n, n), 7.0, dtype=torch.float32, device="cuda")
        F.tabulate(fm, cells[:count].contiguous(), verts,
                   coeffs=coeffs[:count].contiguous() if coeffs is not None else None, out=out[:count],
                   precision="fp32")
        got = out.double().cpu().numpy()
        assert OE.frobenius_rel_error(got[:count], ref[:count]).max() <= FP32_TOL
        assert np.all(got[count] == 7.0)  # the guard cell after the output is untouched
    assert F.status_poll() == 0


def test_bounded_wait_gives_up_and_reports_timeout(F):
    """Failure detection without a fault: a device wait that nothing ends (the probe's
    mbarrier never completes) gives up after its limit, the status word reports
    FLAG_TIMEOUT, and the context stays usable for the next launch."""
    import torch

    assert F.status_poll() == 0
    for polls in (0, 1, 4096):
        F.diag_bounded_wait(polls)
        assert F.status_poll() & F.FLAG_TIMEOUT
    p = _case(3, 2, W.POISSON, 2)
    form = F.Form(W.POISSON, 3, 2)
    A = F.tabulate(form, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64))
    assert F.status_poll() == 0
    assert OE.frobenius_rel_error(A.cpu().numpy(), _oracle(p)).max() <= FP64_TOL


@pytest.mark.parametrize("d,n,q", [(3, 3, 1), (3, 3, 2), (3, 3, 3), (3, 2, 4), (2, 6, 1), (2, 4, 4)])
def test_assemble_pair_matches_the_single_assemblies(F, d, n, q):
    """ffc_assemble_pair(mass, Poisson) in FP32 is one launch; each matrix must equal its own
    ffc_assemble (same contributions: FP64 rounding apart) and the oracle's Algorithm 2.
    The reversed order and FP64 (two launches) give the same matrices."""
    import torch

    p = _case(d, n, W.POISSON, q)
    row_ptr, col, slot_h = F.csr_pattern(p.dofmap, p.n_dof)
    slot = _dev(slot_h, torch.int32)
    cells, verts = _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64)
    fm, fp = F.Form(W.MASS, d, q), F.Form(W.POISSON, d, q)
    gv = M.gather_cell_vertices(p.mesh)
    for prec, tol in (("fp32", FP32_TOL), ("fp64", FP64_TOL)):
        single = []
        for f in (fm, fp):
            v = torch.zeros(col.size, dtype=torch.float64, device="cuda")
            F.assemble(f, cells, verts, slot, v, precision=prec)
            single.append(v)
        vm = torch.zeros(col.size, dtype=torch.float64, device="cuda")
        vp = torch.zeros_like(vm)
        F.assemble_pair(fm, fp, cells, verts, slot, vm, vp, precision=prec)
        wp = torch.zeros_like(vm)
        wm = torch.zeros_like(vm)
        F.assemble_pair(fp, fm, cells, verts, slot, wp, wm, precision=prec)
        assert F.status_poll() == 0
        for got, alt, ref, form in ((vm, wm, single[0], W.MASS), (vp, wp, single[1], W.POISSON)):
            scale = ref.abs().max().item()
            assert (got - ref).abs().max().item() <= 1e-12 * scale
            assert (alt - ref).abs().max().item() <= 1e-12 * scale
            _, _, oracle_val = OA.assemble_csr(OE.element_tensors(form, gv, q), p.dofmap, p.n_dof)
            g = got.cpu().numpy()
            assert np.linalg.norm(g - oracle_val) <= tol * np.linalg.norm(oracle_val)


def test_assemble_pair_arguments(F):
    import torch

    p = _case(3, 2, W.POISSON, 2)
    _, col, slot_h = F.csr_pattern(p.dofmap, p.n_dof)
    slot = _dev(slot_h, torch.int32)
    cells, verts = _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64)
    a = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(F.FFCError) as e:  # one matrix passed twice
        F.assemble_pair(F.Form(W.MASS, 3, 2), F.Form(W.POISSON, 3, 2), cells, verts, slot, a, a)
    assert e.value.code == -1
    with pytest.raises(F.FFCError) as e:  # forms on different spaces
        F.assemble_pair(F.Form(W.MASS, 3, 2), F.Form(W.POISSON, 3, 1), cells, verts, slot, a, b)
    assert e.value.code == -1
    # another pair without coefficients: two assemblies
    F.assemble_pair(F.Form(W.POISSON, 3, 2), F.Form(W.POISSON, 3, 2), cells, verts, slot, a, b, precision="fp32")
    assert torch.equal(a, b)
    assert F.status_poll() == 0


@pytest.mark.parametrize("q", [2, 3])
def test_full_size_pair_assembly(F, q):
    """48^3 x 6 = 663,552 tets, P2 / P3, as the benchmark assembles them: the pair launch's
    mass and Poisson matrices equal the single-form assemblies to FP64 rounding, the mass
    matrix sums to |Omega| = 1 and the Poisson rows sum to zero."""
    import torch

    mesh = W.tet_scalar_mesh(48)
    p = W.make_problem(mesh, W.POISSON, q)
    row_ptr, col, slot_h = _pattern(F, p)
    slot = _dev(slot_h, torch.int32)
    cells, verts = _dev(mesh.cells, torch.int32), _dev(mesh.vertices, torch.float64)
    fm, fp = F.Form(W.MASS, 3, q), F.Form(W.POISSON, 3, q)
    vm = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    vp = torch.zeros_like(vm)
    F.assemble_pair(fm, fp, cells, verts, slot, vm, vp, precision="fp32")
    for f, got in ((fm, vm), (fp, vp)):
        ref = torch.zeros_like(vm)
        F.assemble(f, cells, verts, slot, ref, precision="fp32")
        assert (got - ref).abs().max().item() <= 1e-13 * ref.abs().max().item()
        del ref
    assert F.status_poll() == 0
    assert abs(vm.sum().item() - 1.0) < 1e-6
    rows = torch.repeat_interleave(torch.arange(p.n_dof, device="cuda"),
                                   torch.as_tensor(np.diff(row_ptr), device="cuda"))
    rs = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda").index_add_(0, rows, vp)
    assert rs.abs().max().item() < 1e-5 * vp.abs().max().item()


@pytest.mark.parametrize("prec,alg", [("fp32", "block"), ("fp64", "block"), ("bf16x3", "dense")])
def test_full_size_convection_sampled(F, prec, alg):
    """The vector-P2 convection workload at full size (40^3 x 6 = 384,000 tets), as the
    benchmark tabulates it: several tiles per CTA, so the FP32 block kernel's staging
    buffers rotate across tiles. 500 seeded cells and the last one against the oracle."""
    import torch

    p = W.ns_vp2(40)
    m = p.mesh
    fm = F.Form(W.NS_CONVECTION, 3, 2, algorithm=F.ALG_BLOCK if alg == "block" else F.ALG_DENSE)
    A = F.tabulate(fm, _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64),
                   coeffs=_dev(p.coeffs, torch.float64), precision=prec)
    assert F.status_poll() == 0
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(m.n_elem, 500, replace=False))
    idx[-1] = m.n_elem - 1
    ref = OE.element_tensors(W.NS_CONVECTION, m.vertices[m.cells[idx]], 2, coeffs=p.coeffs[idx])
    got = A[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    err = OE.frobenius_rel_error(got, ref)
    assert err.max() <= (FP64_TOL if prec == "fp64" else FP32_TOL), err.max()


@pytest.mark.parametrize("prec,alg", [("fp32", "block"), ("tf32x3", "dense")])
def test_full_size_elasticity_p3_sampled(F, prec, alg):
    """Elasticity vector P3 on the batched workload's largest mesh size (31^3 x 6 = 178,746
    tets), tabulated as the benchmark times it (FP32 block kernel: 416 threads, two CTAs
    per SM; 3xTF32 tensor cores): 300 seeded cells and the last one against the oracle."""
    import torch

    m = M.unit_cube_tets(31, 0.15, seed=4031)
    fm = F.Form(W.ELASTICITY, 3, 3, algorithm=F.ALG_BLOCK if alg == "block" else F.ALG_DENSE)
    A = F.tabulate(fm, _dev(m.cells, torch.int32), _dev(m.vertices, torch.float64), precision=prec)
    assert F.status_poll() == 0
    rng = np.random.default_rng(12)
    idx = np.sort(rng.choice(m.n_elem, 300, replace=False))
    idx[-1] = m.n_elem - 1
    ref = OE.element_tensors(W.ELASTICITY, m.vertices[m.cells[idx]], 3)
    got = A[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    assert OE.frobenius_rel_error(got, ref).max() <= FP32_TOL
