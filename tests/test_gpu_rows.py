"""Row-owner assembly (ffc_assemble_rows): parity with the oracle's Algorithm 2 on
seeded meshes (triangles and tetrahedra, mass and Poisson, P1-P4, FP64 and FP32), the
exactness of its fixed-point sums (FP32: the correctly rounded sum of the very
contributions the fused kernel adds), determinism, overwrite semantics, edge cases and
errors of the plan, and a sampled oracle check at the full 48^3 x 6 workload."""
import math

import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import mesh as M
from synthetic import workloads as W

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


def _case(d, n, form, q, seed=23, jitter=0.2):
    m = M.unit_square_triangles(n, jitter, seed) if d == 2 else M.unit_cube_tets(n, jitter, seed)
    return W.make_problem(m, form, q, seed=seed)


def _plan(F, p, row_ptr=None, col=None):
    import torch

    if row_ptr is None:
        row_ptr, col, _ = F.csr_pattern(p.dofmap, p.n_dof, with_slots=False)
    plan = F.RowPlan(_dev(p.dofmap, torch.int32), p.n_dof, _dev(row_ptr, torch.int64), _dev(col, torch.int32))
    return plan, row_ptr, col


def _rows(F, p, prec, plan=None):
    import torch

    if plan is None:
        plan, _, _ = _plan(F, p)
    form = F.Form(p.form, p.mesh.dim, p.degree)
    val = torch.full((plan.nnz,), 7.5, dtype=torch.float64, device="cuda")  # overwritten
    F.assemble_rows(form, plan, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64), val,
                    precision=prec)
    return val


CASES = [(2, 7, W.POISSON, 1), (2, 5, W.POISSON, 2), (2, 4, W.MASS, 3), (2, 4, W.POISSON, 4), (2, 3, W.MASS, 4),
         (3, 4, W.MASS, 1), (3, 4, W.POISSON, 1), (3, 3, W.MASS, 2), (3, 3, W.POISSON, 2),
         (3, 3, W.POISSON, 3), (3, 2, W.MASS, 3), (3, 2, W.MASS, 4), (3, 2, W.POISSON, 4)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,n,form,q", CASES)
def test_rows_match_oracle_algorithm2(F, d, n, form, q, prec):
    p = _case(d, n, form, q)
    ref_ptr, ref_col, ref_val = OA.assemble_csr(OE.element_tensors(form, M.gather_cell_vertices(p.mesh), q),
                                                p.dofmap, p.n_dof)
    plan, row_ptr, col = _plan(F, p)
    assert np.array_equal(row_ptr, ref_ptr) and np.array_equal(col, ref_col)
    assert plan.nnz == ref_val.size and plan.max_row == int(np.diff(ref_ptr).max())
    got = _rows(F, p, prec, plan).cpu().numpy()
    assert F.status_poll() == 0
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert np.linalg.norm(got - ref_val) <= tol * np.linalg.norm(ref_val)
    assert np.abs(got - ref_val).max() <= 10 * tol * np.abs(ref_val).max()


@pytest.mark.parametrize("d,n,form,q", [(3, 3, W.POISSON, 2), (3, 2, W.POISSON, 4), (3, 2, W.MASS, 4),
                                        (2, 5, W.POISSON, 3)])
def test_rows_fp32_are_exact_sums_of_the_fused_contributions(F, d, n, form, q):
    """FP32 row-owner assembly computes the same FP32 contributions as ffc_tabulate /
    ffc_assemble (same G_K, same contraction order) and sums them exactly: each entry is
    the correctly rounded exact sum (math.fsum) up to the fixed-point unit, i.e. within
    an ulp plus 2^-44 of the row's sum of |contributions|."""
    import torch

    p = _case(d, n, form, q)
    fm = F.Form(form, d, q)
    A = F.tabulate(fm, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64), precision="fp32")
    contrib = A.double().cpu().numpy().reshape(p.n_elem, -1)
    plan, row_ptr, col = _plan(F, p)
    got = _rows(F, p, "fp32", plan).cpu().numpy()
    assert F.status_poll() == 0
    _, _, slot = F.csr_pattern(p.dofmap, p.n_dof)
    s = slot.reshape(-1)
    v = contrib.reshape(-1)
    order = np.argsort(s, kind="stable")
    s, v = s[order], v[order]
    starts = np.concatenate([[0], np.nonzero(np.diff(s))[0] + 1, [s.size]])
    exact = np.array([math.fsum(v[starts[k]:starts[k + 1]]) for k in range(starts.size - 1)])
    rows = np.repeat(np.arange(p.n_dof), np.diff(row_ptr))
    row_abs = np.zeros(p.n_dof)
    np.add.at(row_abs, np.repeat(p.dofmap.reshape(-1), p.n_local), np.abs(contrib.reshape(-1)))
    tol = np.spacing(np.abs(exact)) + 2.0 ** -44 * row_abs[rows]
    assert np.all(np.abs(got - exact) <= tol)
    assert np.mean(got == exact) > 0.5  # most entries are the correctly rounded sum itself


def test_rows_are_deterministic_and_overwrite(F):
    import torch

    p = _case(3, 3, W.POISSON, 3)
    plan, _, _ = _plan(F, p)
    a = _rows(F, p, "fp32", plan)
    b = _rows(F, p, "fp32", plan)
    assert torch.equal(a, b)  # bitwise, independent of scheduling
    form = F.Form(W.POISSON, 3, 3)
    c = torch.full_like(a, float("nan"))
    F.assemble_rows(form, plan, _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64), c,
                    precision="fp32")
    assert torch.equal(a, c)
    assert F.status_poll() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rows_agree_with_the_atomic_assembly(F, prec):
    import torch

    p = _case(3, 3, W.POISSON, 3)
    plan, row_ptr, col = _plan(F, p)
    got = _rows(F, p, prec, plan)
    _, _, slot = F.csr_pattern(p.dofmap, p.n_dof)
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble(F.Form(W.POISSON, 3, 3), _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64),
               _dev(slot, torch.int32), val, precision=prec)
    assert F.status_poll() == 0
    # the same contributions summed in two orders: FP64 rounding apart
    assert (got - val).abs().max().item() <= 1e-13 * val.abs().max().item()


def test_rows_edge_cases(F):
    import torch

    # a single cell; and a dof that no cell touches (an empty row)
    m = M.unit_cube_tets(1, 0.0, 0)
    p = W.make_problem(m, W.POISSON, 2)
    one = W.FormProblem(M.SimplexMesh(m.vertices, m.cells[:1], m.lattice, m.n), W.POISSON, 2, p.dofmap[:1], p.n_dof)
    dm = one.dofmap
    row_ptr, col, _ = F.csr_pattern(dm, p.n_dof, with_slots=False)
    plan, _, _ = _plan(F, one, row_ptr, col)
    got = _rows(F, one, "fp64", plan).cpu().numpy()
    ref = OE.element_tensors(W.POISSON, M.gather_cell_vertices(one.mesh), 2)[0]
    _, _, ref_val = OA.assemble_csr(ref[None], dm, p.n_dof)
    assert np.abs(got - ref_val).max() <= FP64_TOL * np.abs(ref_val).max()
    assert plan.max_incidence == 1
    # no cells: an empty pattern, nothing launched
    empty = W.FormProblem(M.SimplexMesh(m.vertices, m.cells[:0], m.lattice, m.n), W.POISSON, 2, p.dofmap[:0], p.n_dof)
    rp0 = np.zeros(p.n_dof + 1, dtype=np.int64)
    plan0 = F.RowPlan(torch.zeros((0, 10), dtype=torch.int32, device="cuda"), p.n_dof,
                      _dev(rp0, torch.int64), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert plan0.nnz == 0 and plan0.max_row == 0
    _rows(F, empty, "fp32", plan0)
    assert F.status_poll() == 0


def test_rows_plan_errors(F):
    import torch

    p = _case(3, 2, W.POISSON, 2)
    row_ptr, col, _ = F.csr_pattern(p.dofmap, p.n_dof, with_slots=False)
    dm = _dev(p.dofmap, torch.int32)
    # a dof id out of range
    bad = p.dofmap.copy()
    bad[3, 4] = p.n_dof + 5
    with pytest.raises(F.FFCError) as e:
        F.RowPlan(_dev(bad, torch.int32), p.n_dof, _dev(row_ptr, torch.int64), _dev(col, torch.int32))
    assert e.value.code == -6
    # a pair missing from the pattern (drop the first entry of row 0)
    rp = row_ptr.copy()
    rp[1:] -= 1
    with pytest.raises(F.FFCError) as e:
        F.RowPlan(dm, p.n_dof, _dev(rp, torch.int64), _dev(col[1:], torch.int32))
    assert e.value.code == -6
    # a row_ptr that is not monotone
    rp = row_ptr.copy()
    rp[5] = rp[7]
    with pytest.raises(F.FFCError) as e:
        F.RowPlan(dm, p.n_dof, _dev(rp, torch.int64), _dev(col, torch.int32))
    assert e.value.code == -1
    # a form with another number of local dofs, and a form the kernel does not carry
    plan = F.RowPlan(dm, p.n_dof, _dev(row_ptr, torch.int64), _dev(col, torch.int32))
    cells, verts = _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64)
    val = torch.zeros(plan.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FFCError) as e:
        F.assemble_rows(F.Form(W.POISSON, 3, 1), plan, cells, verts, val)
    assert e.value.code == -1
    with pytest.raises(F.FFCError) as e:
        F.assemble_rows(F.Form(W.SOURCE, 3, 2), plan, cells, verts, val)
    assert e.value.code == -5
    assert F.status_poll() == 0


def test_rows_of_a_degenerate_cell_are_nan_and_flagged(F):
    import torch

    p = _case(3, 2, W.POISSON, 1)
    verts = p.mesh.vertices.copy()
    c = p.mesh.cells[5]
    verts[c[3]] = verts[c[0]]  # cell 5 collapses to a triangle (det J = 0)
    plan, row_ptr, _ = _plan(F, p)
    val = torch.zeros(plan.nnz, dtype=torch.float64, device="cuda")
    F.assemble_rows(F.Form(W.POISSON, 3, 1), plan, _dev(p.mesh.cells, torch.int32), _dev(verts, torch.float64),
                    val, precision="fp64")
    assert F.status_poll() & F.FLAG_DEGENERATE
    v = val.cpu().numpy()
    rows = np.repeat(np.arange(p.n_dof), np.diff(row_ptr))
    bad_rows = set(p.dofmap[5].tolist())
    in_bad = np.isin(rows, list(bad_rows))
    assert np.all(np.isnan(v[in_bad]))


def _sampled_rows_oracle(mesh, dofmap, form, q, row_ptr, col, rows_sel):
    """Oracle values of the selected rows: Algorithm 2 restricted to the cells that hold
    each row's dof (every contribution to the row comes from them)."""
    sel = set(int(r) for r in rows_sel)
    cells = np.nonzero(np.isin(dofmap, list(sel)).any(axis=1))[0]
    AK = OE.element_tensors(form, mesh.vertices[mesh.cells[cells]], q)
    out = {}
    for k, e in enumerate(cells):
        for i1, r in enumerate(dofmap[e]):
            if int(r) not in sel:
                continue
            row = out.setdefault(int(r), {})
            for i2, cj in enumerate(dofmap[e]):
                row[int(cj)] = row.get(int(cj), 0.0) + AK[k, i1, i2]
    return out


@pytest.mark.parametrize("form,q", [(W.MASS, 4), (W.POISSON, 4), (W.POISSON, 2)])
def test_full_size_rows_sampled_against_the_oracle(F, form, q):
    """48^3 x 6 = 663,552 tets, as the benchmark runs it (FP32): 64 seeded rows checked
    entry by entry against the oracle, the whole matrix through its invariants (total
    mass = |Omega|, Poisson row sums = 0) and against the atomic fused assembly."""
    import torch

    mesh = W.tet_scalar_mesh(48)
    p = W.make_problem(mesh, form, q)
    row_ptr, col, _ = F.csr_pattern(p.dofmap, p.n_dof, with_slots=False)
    plan, _, _ = _plan(F, p, row_ptr, col)
    fm = F.Form(form, 3, q)
    cells, verts = _dev(mesh.cells, torch.int32), _dev(mesh.vertices, torch.float64)
    val = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    F.assemble_rows(fm, plan, cells, verts, val, precision="fp32")
    assert F.status_poll() == 0
    rng = np.random.default_rng(7)
    rows_sel = np.sort(rng.choice(p.n_dof, 64, replace=False))
    rows_sel[-1] = p.n_dof - 1
    ref = _sampled_rows_oracle(mesh, p.dofmap, form, q, row_ptr, col, rows_sel)
    v = val.cpu().numpy()
    for r in rows_sel:
        seg = slice(row_ptr[r], row_ptr[r + 1])
        want = np.array([ref[int(r)][int(c)] for c in col[seg]])
        assert np.linalg.norm(v[seg] - want) <= FP32_TOL * np.linalg.norm(want)
    if form == W.MASS:
        assert abs(v.sum() - 1.0) < 1e-6
    else:
        rows = np.repeat(np.arange(p.n_dof), np.diff(row_ptr))
        rs = np.bincount(rows, weights=v, minlength=p.n_dof)
        assert np.abs(rs).max() < 1e-5 * np.abs(v).max()
    del v
    if form != W.POISSON or q != 4:
        return
    _, _, slot = F.csr_pattern(p.dofmap, p.n_dof)
    ref_val = torch.zeros_like(val)
    F.assemble(fm, cells, verts, _dev(slot, torch.int32), ref_val, precision="fp32")
    assert F.status_poll() == 0
    assert (val - ref_val).abs().max().item() <= 1e-13 * ref_val.abs().max().item()
