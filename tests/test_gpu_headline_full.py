"""The benchmark's headline step checked at its full size: 48^3 x 6 = 663,552 Kuhn
tetrahedra, mass and Poisson with P1..P4, FP32 contraction and FP64 CSR values, run
exactly as ``bench.py`` runs it (the same workload builder and the same step function).

Two kinds of checks on all eight assembled matrices:

* properties that hold at any size: total mass = |Omega| = 1, zero row sums of the
  Poisson matrices (relative to each row's sum of |entries|), and the energies
  u^T A u of interpolated polynomials (u = x: mass 1/3, Poisson 1; u = x^2 for q >= 2:
  mass 1/5, Poisson 4/3), which Lagrange P_q reproduces exactly;
* a seeded sample of at least 200 whole CSR rows per matrix against the oracle's
  Algorithm 2 (Section 2.2) over the cells incident to each row: the row's columns bit
  for bit, each value within 1e-6 of the row's sum of |contributions| (the stated
  mixed-precision target).

Also here: configuration 1 at its stated size (P1 Poisson on 64 x 64 x 2 triangles,
FP64), every element tensor and the assembled CSR matrix against the oracle.
"""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import dofmap as D
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ROW_TOL = 1e-6       # mixed-precision target, relative to the row's sum of |contributions|
ROWS_PER_MATRIX = 200


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    assert torch.cuda.is_available()
    return F


@pytest.fixture(scope="module")
def headline(F):
    import torch

    import bench

    dev = torch.device("cuda", 0)
    ctx = bench.build_workload(F, 48, dev)
    bench.run_headline_step(F, ctx, "fp32")
    torch.cuda.synchronize()
    assert F.status_poll() == 0
    return ctx


def _dof_coordinates(ctx, q, dofmap, n_dof):
    """Physical position of every global dof (the lattice point of a cell mapped affinely)."""
    import torch

    lat = torch.as_tensor(D.local_lattice(3, q), dtype=torch.float64, device="cuda") / q  # [n, 4]
    xc = ctx["verts"][ctx["cells"].long()]  # [E, 4, 3]
    pos = torch.einsum("nj,ejx->enx", lat, xc).reshape(-1, 3)
    out = torch.zeros((n_dof, 3), dtype=torch.float64, device="cuda")
    out[torch.as_tensor(dofmap, device="cuda").long().reshape(-1)] = pos
    return out


def _csr(ctx, pr):
    import torch

    pat = ctx["patterns"][pr["q"]]
    crow = torch.as_tensor(pat["row_ptr"], device="cuda")
    col = torch.as_tensor(pat["col"], device="cuda").long()
    return torch.sparse_csr_tensor(crow, col, pr["val"], size=(pat["n_dof"], pat["n_dof"]))


def test_headline_matrices_invariants(headline):
    import torch

    ctx = headline
    for pr in ctx["problems"]:
        q, pat = pr["q"], ctx["patterns"][pr["q"]]
        val = pr["val"]
        assert bool(torch.isfinite(val).all())
        if pr["form"] == W.MASS:
            assert abs(val.sum().item() - 1.0) <= 1e-6, f"mass P{q}: total mass"
        else:
            rows = torch.repeat_interleave(torch.arange(pat["n_dof"], device="cuda"),
                                           torch.as_tensor(np.diff(pat["row_ptr"]), device="cuda"))
            rs = torch.zeros(pat["n_dof"], dtype=torch.float64, device="cuda").index_add_(0, rows, val)
            ra = torch.zeros(pat["n_dof"], dtype=torch.float64, device="cuda").index_add_(0, rows, val.abs())
            assert (rs.abs() <= ROW_TOL * ra).all(), f"Poisson P{q}: row sums"
            del rows, rs, ra
        A = _csr(ctx, pr)
        absA = _csr(ctx, {"q": q, "val": val.abs()})
        x = _dof_coordinates(ctx, q, pat["dofmap"], pat["n_dof"])
        fields = [(x[:, 0], 1.0 / 3.0 if pr["form"] == W.MASS else 1.0)]
        if q >= 2:
            fields.append((x[:, 0] ** 2, 1.0 / 5.0 if pr["form"] == W.MASS else 4.0 / 3.0))
        for u, exact in fields:
            energy = torch.dot(u, (A @ u.unsqueeze(1)).squeeze(1)).item()
            # FP32 contributions carry ~1e-7 relative error each; the quadratic form of the
            # stiffness matrix cancels (zero row sums), so the bound is relative to |u|^T |A| |u|
            scale = torch.dot(u.abs(), (absA @ u.abs().unsqueeze(1)).squeeze(1)).item()
            assert abs(energy - exact) <= ROW_TOL * scale, f"form {pr['form']} P{q}: u^T A u {energy} vs {exact}"
            if pr["form"] == W.MASS:
                assert abs(energy - exact) <= ROW_TOL * exact
        del A, absA, x
        torch.cuda.empty_cache()


def _sample_rows(n_dof, q, n, rng):
    side = round(n_dof ** (1.0 / 3.0))
    assert side ** 3 == n_dof
    ijk = rng.integers(1, side - 1, size=(40, 3)) // q * q  # interior vertex dofs (24 cells each)
    vertex_rows = (ijk[:, 0] * side + ijk[:, 1]) * side + ijk[:, 2]
    picks = np.concatenate([[0, n_dof - 1, n_dof // 2], vertex_rows, rng.choice(n_dof, n, replace=False)])
    return np.unique(picks)


def test_headline_rows_against_oracle(headline):
    """At least 200 whole rows of each of the eight matrices against Algorithm 2 of the
    oracle over the rows' incident cells (element tensors by quadrature on each cell)."""
    ctx = headline
    mesh = ctx["mesh"]
    rng = np.random.default_rng(20261203)
    for pr in ctx["problems"]:
        q, pat = pr["q"], ctx["patterns"][pr["q"]]
        dofmap, n_dof, row_ptr, col = pat["dofmap"], pat["n_dof"], pat["row_ptr"], pat["col"]
        rows = _sample_rows(n_dof, q, ROWS_PER_MATRIX, rng)
        assert rows.size >= ROWS_PER_MATRIX
        hit = np.isin(dofmap, rows)
        cells = np.nonzero(hit.any(axis=1))[0]
        ref_K = OE.element_tensors(pr["form"], mesh.vertices[mesh.cells[cells]], q)
        val = pr["val"].cpu().numpy()
        for r in rows:
            es, i1s = np.nonzero(dofmap[cells] == r)
            ref = {}
            bound = 0.0
            for e, i1 in zip(es, i1s):
                for i2 in range(dofmap.shape[1]):
                    c = int(dofmap[cells[e], i2])
                    v = ref_K[e, i1, i2]
                    ref[c] = ref.get(c, 0.0) + v
                    bound += abs(v)
            lo, hi = row_ptr[r], row_ptr[r + 1]
            cols = col[lo:hi]
            assert np.array_equal(cols, np.array(sorted(ref), dtype=cols.dtype)), f"row {r}: pattern"
            want = np.array([ref[int(c)] for c in cols])
            err = np.abs(val[lo:hi] - want).max()
            assert err <= ROW_TOL * bound, f"form {pr['form']} P{q} row {r}: {err / bound:.3e}"


def test_config1_p1_triangles_fp64(F):
    """P1 Poisson on the unit square, 64 x 64 x 2 triangles (8192 cells, 4225 vertices),
    jitter 0.2h: every element tensor at 1e-12 and the assembled matrix (fused atomic
    assembly and row-owner assembly) against the oracle's Algorithm 2."""
    import torch

    p = W.poisson_p1_tri()
    assert p.n_elem == 8192 and p.mesh.n_vert == 4225
    cells = torch.as_tensor(p.mesh.cells, device="cuda")
    verts = torch.as_tensor(p.mesh.vertices, device="cuda")
    fm = F.Form(F.POISSON, F.TRIANGLE, 1)
    A = F.tabulate(fm, cells, verts, precision="fp64")
    assert F.status_poll() == 0
    ref = OE.element_tensors(W.POISSON, M.gather_cell_vertices(p.mesh), 1)
    assert OE.frobenius_rel_error(A.cpu().numpy(), ref).max() <= 1e-12
    ref_ptr, ref_col, ref_val = OA.assemble_csr(ref, p.dofmap, p.n_dof)
    row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
    assert np.array_equal(row_ptr, ref_ptr) and np.array_equal(col, ref_col) and col.size == 29057
    _, _, bound = OA.assemble_csr(np.abs(ref), p.dofmap, p.n_dof)
    rows = np.repeat(np.arange(p.n_dof), np.diff(row_ptr))
    row_bound = np.bincount(rows, bound, p.n_dof)[rows]
    val = torch.zeros(col.size, dtype=torch.float64, device="cuda")
    F.assemble(fm, cells, verts, torch.as_tensor(slot, device="cuda"), val, precision="fp64")
    assert F.status_poll() == 0
    assert (np.abs(val.cpu().numpy() - ref_val) <= 1e-12 * row_bound).all()
    plan = F.RowPlan(torch.as_tensor(p.dofmap, device="cuda"), p.n_dof, torch.as_tensor(row_ptr, device="cuda"),
                     torch.as_tensor(col, device="cuda"))
    for prec, tol in (("fp64", 1e-12), ("fp32", ROW_TOL)):
        out = torch.full((col.size,), float("nan"), dtype=torch.float64, device="cuda")
        F.assemble_rows(fm, plan, cells, verts, out, precision=prec)
        assert F.status_poll() == 0
        assert (np.abs(out.cpu().numpy() - ref_val) <= tol * row_bound).all(), prec
