"""The batched heterogeneous launch (one persistent kernel over many problems, a
global tile queue, tuned tile variant, CUDA-graph replay) against the oracle's
Algorithm-2 assembly of every problem."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-6


@pytest.fixture(scope="module")
def F():
    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    return F


def _items(F, specs):
    import torch

    items, refs = [], []
    for k, (form, q, n) in enumerate(specs):
        m = M.unit_cube_tets(n, 0.15, seed=40 + k)
        p = W.make_problem(m, form, q, seed=40 + k)
        row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
        _, _, ref = OA.assemble_csr(OE.element_tensors(form, M.gather_cell_vertices(m), q), p.dofmap, p.n_dof)
        items.append({"form": F.Form(form, F.TETRAHEDRON, q),
                      "cells": torch.as_tensor(m.cells, device="cuda"),
                      "vertices": torch.as_tensor(m.vertices, device="cuda"),
                      "slot": torch.as_tensor(slot, device="cuda"),
                      "csr_val": torch.full((col.size,), 7.0, dtype=torch.float64, device="cuda")})
        refs.append(ref)
    return items, refs


def _check(items, refs):
    for it, ref in zip(items, refs):
        got = it["csr_val"].cpu().numpy()
        assert np.linalg.norm(got - ref) <= FP32_TOL * np.linalg.norm(ref)


SPECS = [(W.ELASTICITY, 1, 3), (W.ELASTICITY, 2, 2), (W.ELASTICITY, 3, 2), (W.POISSON, 2, 3),
         (W.POISSON, 1, 4), (W.MASS, 1, 2), (W.ELASTICITY, 2, 1), (W.POISSON, 2, 1)]


def test_batch_matches_oracle_plain_tuned_and_graph(F):
    items, refs = _items(F, SPECS)
    b = F.Batch(items, zero_csr=True)
    info = b.info()
    assert info["items"] == len(SPECS) and info["tiles"] > 0
    b.run(graph=False)
    assert F.status_poll() == 0
    _check(items, refs)  # zero_csr replaced the 7.0 fill
    ke = b.tune()
    assert ke in (16, 32, 64, 128)
    for _ in range(2):
        b.run(graph=True)
        assert F.status_poll() == 0
        _check(items, refs)  # replays start from zeroed values each time
    b.close()


def test_batch_accumulates_without_zeroing(F):
    items, refs = _items(F, SPECS[:3])
    for it in items:
        it["csr_val"].zero_()
    b = F.Batch(items, zero_csr=False)
    b.run()
    b.run()
    assert F.status_poll() == 0
    _check(items, [2 * r for r in refs])


def test_batch_rejects_forms_it_does_not_carry(F):
    items, _ = _items(F, [(W.POISSON, 2, 1)])
    items[0]["form"] = F.Form(W.POISSON, F.TETRAHEDRON, 4)
    n = 35
    import torch
    items[0]["slot"] = torch.zeros((items[0]["cells"].shape[0], n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FFCError) as e:
        F.Batch(items)
    assert e.value.code == -5
