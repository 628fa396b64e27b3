"""The batched workload at full size (32 meshes, 1.77 M tets, elasticity vP1-vP3 and
Poisson P2 in one persistent launch), checked through properties of every assembled
matrix that hold at any size: rigid-body modes lie in the kernel of each elasticity
matrix, a linear displacement u = B x has energy int 2 mu |sym B|^2 + lambda (tr B)^2
over the unit cube, Poisson rows sum to zero and u = x^2 has energy 4/3.

The mixed-precision bar is per entry (relative 1e-6), so each quadratic-form check is
bounded by 1e-6 |u|^T |A| |u| with |A| the entrywise absolute matrix: the energies cancel
strongly (A annihilates constants), which a relative bound on the energy itself ignores."""
import numpy as np
import pytest

from synthetic import mesh as M
from synthetic import workloads as W
from synthetic.dofmap import local_lattice

pytestmark = pytest.mark.gpu
ENTRY_TOL = 1e-6  # FP32 contraction, FP64 accumulation


def _dof_coords(p):
    """Coordinates of every global dof (lattice points of the jittered cells)."""
    d = p.mesh.dim
    lam = local_lattice(d, p.degree).astype(float) / p.degree
    x = np.einsum("kj,ejx->ekx", lam, M.gather_cell_vertices(p.mesh))  # [E, n_s, d]
    ns = lam.shape[0]
    scalar_ids = p.dofmap[:, :ns] if p.form == W.POISSON else p.dofmap[:, :ns] // d
    n_scalar = p.n_dof if p.form == W.POISSON else p.n_dof // d
    out = np.zeros((n_scalar, d))
    out[scalar_ids.reshape(-1)] = x.reshape(-1, d)
    return out


def test_batched_workload_full_size_properties():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    probs = W.batched()
    items, csr = [], []
    for pb in probs:
        row_ptr, col, slot = F.csr_pattern(pb.dofmap, pb.n_dof)
        items.append({"form": F.Form(pb.form, F.TETRAHEDRON, pb.degree),
                      "cells": torch.as_tensor(pb.mesh.cells, device="cuda"),
                      "vertices": torch.as_tensor(pb.mesh.vertices, device="cuda"),
                      "slot": torch.as_tensor(slot, device="cuda"),
                      "csr_val": torch.zeros(col.size, dtype=torch.float64, device="cuda")})
        csr.append((torch.as_tensor(row_ptr, device="cuda"), torch.as_tensor(col.astype(np.int64), device="cuda")))
        del slot
    b = F.Batch(items, zero_csr=True)
    b.tune()
    b.run(graph=True)
    assert F.status_poll() == 0
    Bmat = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.6], [0.25, 0.05, -0.1]])
    S = 0.5 * (Bmat + Bmat.T)
    for pb, it, (rp, cl) in zip(probs, items, csr):
        A = torch.sparse_csr_tensor(rp, cl, it["csr_val"], size=(pb.n_dof, pb.n_dof))
        Aabs = torch.sparse_csr_tensor(rp, cl, it["csr_val"].abs(), size=(pb.n_dof, pb.n_dof))

        def bound(u):
            return ENTRY_TOL * (u.abs() @ (Aabs @ u.abs())).item()

        X = _dof_coords(pb)
        scale = it["csr_val"].abs().max().item()
        if pb.form == W.POISSON:
            one = torch.ones(pb.n_dof, dtype=torch.float64, device="cuda")
            assert bool(((A @ one).abs() <= ENTRY_TOL * (Aabs @ one) + 1e-300).all())
            u = torch.as_tensor(X[:, 0] ** 2, device="cuda")
            assert abs((u @ (A @ u)).item() - 4.0 / 3.0) <= bound(u)
        else:
            for mode in (lambda x: np.stack([np.ones(len(x)), 0 * x[:, 0], 0 * x[:, 0]], 1),
                         lambda x: np.stack([-x[:, 1], x[:, 0], 0 * x[:, 0]], 1),
                         lambda x: np.stack([0 * x[:, 0], -x[:, 2], x[:, 1]], 1)):
                u = torch.as_tensor(mode(X).reshape(-1), device="cuda")  # interleaved global order
                r = A @ u
                assert bool((r.abs() <= ENTRY_TOL * (Aabs @ u.abs()) + 1e-300).all()), (pb.degree, scale)
            u = torch.as_tensor((X @ Bmat.T).reshape(-1), device="cuda")
            energy = (u @ (A @ u)).item()
            assert abs(energy - (2 * np.sum(S * S) + 1.25 * np.trace(Bmat) ** 2)) <= bound(u)
