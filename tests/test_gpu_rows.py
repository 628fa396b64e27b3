"""Row-owner assembly (ffc_assemble_rows): parity with the oracle's Algorithm 2 on
seeded meshes (triangles and tetrahedra, mass and Poisson, P1-P4, FP64 and FP32), the
accuracy of its fixed-point sums (FP32: the very contributions the fused kernel adds,
summed in 31-bit fixed point), determinism, overwrite semantics, edge cases and
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
    ffc_assemble (same G_K, same contraction order) and sums them in 31-bit fixed point:
    the unit of a chunk is u = 2^(eb - 31) with 2^(eb - 2) < B <= 2^(eb - 1), B the
    chunk's bound (largest a0max[i1] * sum|G_K| of its pairs times the most pairs of a
    row), and each contribution is rounded to the nearest multiple of u, off by at most
    u / 2 < 2^-30 B, so each entry is within m * 2^-30 * B of the exact sum (math.fsum) of
    its m contributions, plus the final rounding to FP64. G_K is recovered from the FP32
    element tensors by least squares against the reference tensor, which also checks the
    tensor representation A = A0 : G."""
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
    m = np.diff(starts)
    # the bound B of every chunk is at most the global one
    A0 = fm.reference_tensor()  # [n * n, n_alpha]
    G, *_ = np.linalg.lstsq(A0, contrib.T, rcond=None)  # [n_alpha, n_elem]
    assert np.abs(A0 @ G - contrib.T).max() <= 1e-5 * np.abs(contrib).max()
    a0max = np.abs(A0).reshape(p.n_local, -1).max(axis=1)
    incidence = np.bincount(p.dofmap.reshape(-1), minlength=p.n_dof).max()
    # the kernel bounds Poisson contributions with the symmetric reference tensor (the
    # off-diagonal columns summed, entries up to twice those of the 9-column A0) and the
    # six |G| entries (each off-diagonal once): at most twice this product
    sym = 2.0 if form == W.POISSON else 1.0
    B = sym * a0max.max() * np.abs(G).sum(axis=0).max() * incidence * (1 + 1e-4)
    tol = np.spacing(np.abs(exact)) + m * 2.0 ** -30 * B
    assert np.all(np.abs(got - exact) <= tol)


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
    # the same contributions summed two ways: FP64 atomics against fixed point with 63
    # bits (FP64 path; rounding apart) or 31 bits (FP32 path; each contribution rounded
    # to 2^-30 of its chunk's bound, the per-entry bound checked exactly by
    # test_rows_fp32_are_exact_sums_of_the_fused_contributions)
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert (got - val).abs().max().item() <= tol * val.abs().max().item()


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
    # FP64 atomics against 31-bit fixed point (each contribution rounded to 2^-30 of its
    # chunk's bound)
    assert (val - ref_val).abs().max().item() <= 1e-5 * ref_val.abs().max().item()


@pytest.mark.parametrize("d,n,q", [(3, 3, 1), (3, 3, 2), (3, 2, 3), (3, 2, 4), (2, 5, 2), (2, 4, 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rows_pair_equals_the_single_form_passes(F, d, n, q, prec):
    """ffc_assemble_rows_pair (mass and Poisson in one pass over the plan) writes, bit for
    bit, what two ffc_assemble_rows calls write, in either argument order."""
    import torch

    p = _case(d, n, W.POISSON, q)
    plan, _, _ = _plan(F, p)
    cells, verts = _dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64)
    fm, fp = F.Form(W.MASS, d, q), F.Form(W.POISSON, d, q)
    m1 = torch.full((plan.nnz,), 3.0, dtype=torch.float64, device="cuda")
    p1 = torch.full_like(m1, 3.0)
    F.assemble_rows(fm, plan, cells, verts, m1, precision=prec)
    F.assemble_rows(fp, plan, cells, verts, p1, precision=prec)
    m2, p2 = torch.full_like(m1, float("nan")), torch.full_like(m1, float("nan"))
    F.assemble_rows_pair(fm, fp, plan, cells, verts, m2, p2, precision=prec)
    m3, p3 = torch.full_like(m1, float("nan")), torch.full_like(m1, float("nan"))
    F.assemble_rows_pair(fp, fm, plan, cells, verts, p3, m3, precision=prec)
    assert F.status_poll() == 0
    assert torch.equal(m1, m2) and torch.equal(p1, p2) and torch.equal(m1, m3) and torch.equal(p1, p3)


def test_rows_plan_layout_and_limits(F):
    """The plan's chunk layout, and the limits of a row: more than 4096 entries or more
    than the chunk's pair budget is refused with FFC_EINVAL before any launch."""
    import torch

    p = _case(3, 3, W.POISSON, 4)
    plan, row_ptr, _ = _plan(F, p)
    assert plan.n_chunks >= 1 and 0 < plan.max_chunk_values <= 4096 and 0 < plan.max_chunk_pairs <= 512
    assert plan.max_region_bytes >= 4 * plan.max_chunk_pairs * (1 + p.n_local // 2)
    assert plan.device_bytes > 2 * p.n_elem * p.n_local ** 2
    # a star: dof 0 shared by 1400 cells (row 0 has 4201 entries and 1400 pairs)
    E = 1400
    dm = np.zeros((E, 4), dtype=np.int32)
    dm[:, 1:] = 1 + np.arange(3 * E, dtype=np.int32).reshape(E, 3)
    rp, col, _ = F.csr_pattern(dm, 3 * E + 1, with_slots=False)
    with pytest.raises(F.FFCError) as e:
        F.RowPlan(_dev(dm, torch.int32), 3 * E + 1, _dev(rp, torch.int64), _dev(col, torch.int32))
    assert e.value.code == -1
