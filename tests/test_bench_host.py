"""Host logic of bench.py that needs no GPU: the launch list of the headline step (which
problems share an ffc_assemble_pair or ffc_assemble_rows_pair launch), the kernels each
launch starts, and the algorithmic byte count of a launch."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _ctx():
    nnz = {1: 17, 2: 258, 3: 1460, 4: 5361}  # the 48^3 x 6 patterns' nnz in units of 1e5
    probs = [{"form": f, "q": q, "n_local": (q + 1) * (q + 2) * (q + 3) // 6, "nnz": nnz[q]}
             for q in (1, 2, 3, 4) for f in (0, 1)]

    class Mesh:
        n_elem, n_vert = 10, 7

    return {"problems": probs, "mesh": Mesh()}


def test_launch_list_pairs_the_requested_degrees():
    ctx = _ctx()
    ll = bench.launch_list(ctx, {1, 2, 3})
    # alternately the smallest and the largest remaining launch (a pair counts both matrices)
    assert [lab for lab, _, _ in ll] == ["mass+poisson_p1", "poisson_p4", "mass+poisson_p2", "mass_p4",
                                         "mass+poisson_p3"]
    assert [ks for _, ks, _ in ll] == [[0, 1], [7], [2, 3], [6], [4, 5]]
    assert [kind for _, _, kind in ll] == ["pair", "single", "pair", "single", "pair"]
    # every problem exactly once
    assert sorted(sum((ks for _, ks, _ in ll), [])) == list(range(8))
    assert sorted(ks[0] for _, ks, _ in bench.launch_list(ctx, set())) == list(range(8))
    assert len(bench.launch_list(ctx, {1, 2, 3, 4})) == 4


def test_launch_list_of_the_headline_step():
    """P3 and P4 by the row-owner pair, P1 and P2 by the atomic pair."""
    ctx = _ctx()
    ll = bench.launch_list(ctx, {1, 2, 3}, {3, 4})
    assert [(lab, kind) for lab, _, kind in ll] == [("mass+poisson_p1", "pair"), ("rows_mass+poisson_p4", "rows"),
                                                    ("mass+poisson_p2", "pair"), ("rows_mass+poisson_p3", "rows")]
    assert sorted(sum((ks for _, ks, _ in ll), [])) == list(range(8))
    # geometry + assembly per row-owner call (FP64: per form), one fused kernel per atomic call
    assert sum(bench.kernels_of(e, "fp32") for e in ll) == 2 + 2 + 1 + 1
    assert sum(bench.kernels_of(e, "fp64") for e in ll) == 4 + 4 + 2 + 2


def test_launch_list_rejects_a_problem_order_it_cannot_pair():
    ctx = _ctx()
    ctx["problems"][0], ctx["problems"][1] = ctx["problems"][1], ctx["problems"][0]
    with pytest.raises(AssertionError):
        bench.launch_list(ctx, {1})


def test_algorithmic_bytes_count_the_shared_inputs_once():
    ctx = _ctx()
    one = bench.alg_bytes_assemble(ctx, [ctx["problems"][6]])
    two = bench.alg_bytes_assemble(ctx, ctx["problems"][6:8])
    # cells, vertices and the dof map once, CSR values read and written once per matrix
    assert one == 10 * 16 + 7 * 24 + 10 * 4 * 35 + 16 * 5361
    assert two - one == 16 * 5361
    # the row-owner launch writes each value once and reads none
    rows = bench.alg_bytes_assemble(ctx, ctx["problems"][6:8], "rows")
    assert rows == 10 * 16 + 7 * 24 + 10 * 4 * 35 + 2 * 8 * 5361
