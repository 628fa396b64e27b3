"""The adjoint kernel (dL/dA_K -> dL/dG_K -> dL/dvertices) behind torch.autograd,
for L = sum_K u_K^T A^K v_K (Poisson): against the oracle's continuous shape
derivative and against central finite differences of the GPU forward pass."""
import numpy as np
import pytest

from oracle import shape as OS
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    return F


def _objective_grad(F, p, u, v):
    import torch

    from paper_1112_0402_gb300.autograd import element_tensors

    form = F.Form(F.POISSON, p.mesh.dim, p.degree)
    verts = torch.as_tensor(p.mesh.vertices, device="cuda").requires_grad_(True)
    cells = torch.as_tensor(p.mesh.cells, device="cuda")
    dm = torch.as_tensor(p.dofmap.astype(np.int64), device="cuda")
    uK = torch.as_tensor(u, device="cuda")[dm]
    vK = torch.as_tensor(v, device="cuda")[dm]
    A = element_tensors(form, cells, verts)
    L = torch.einsum("ei,eij,ej->", uK, A, vK)
    L.backward()
    assert F.status_poll() == 0
    return float(L.item()), verts.grad.cpu().numpy(), form


@pytest.mark.parametrize("d,n,q", [(3, 2, 1), (3, 3, 2), (3, 2, 3), (3, 1, 4), (2, 4, 2)])
def test_adjoint_matches_oracle_shape_derivative(F, d, n, q):
    m = M.unit_cube_tets(n, 0.15, seed=8) if d == 3 else M.unit_square_triangles(n, 0.15, seed=8)
    p = W.make_problem(m, W.POISSON, q)
    rng = np.random.default_rng(21)
    u = rng.standard_normal(p.n_dof)
    v = rng.standard_normal(p.n_dof)
    L, g, _ = _objective_grad(F, p, u, v)
    ref = OS.poisson_shape_gradient(m.vertices, m.cells, q, p.dofmap, u, v)
    assert abs(L - OS.poisson_objective(m.vertices, m.cells, q, p.dofmap, u, v)) <= 1e-12 * abs(L) + 1e-12
    assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


def _fd_sample(F, p, u, v, coords, h=1e-6):
    """Central differences of L at sampled (vertex, component) pairs, recomputing only
    the cells incident to each vertex (one batched GPU forward for all samples)."""
    import torch

    m = p.mesh
    form = F.Form(F.POISSON, m.dim, p.degree)
    inc = [[] for _ in range(m.n_vert)]
    for e, c in enumerate(m.cells):
        for vid in c:
            inc[vid].append(e)
    all_cells, all_verts, owner, sign = [], [], [], []
    base = 0
    for k, (vid, comp) in enumerate(coords):
        es = np.array(inc[vid])
        local_ids, local_cells = np.unique(m.cells[es], return_inverse=True)
        local_cells = local_cells.reshape(-1, m.dim + 1)
        for sgn in (+1, -1):
            X = m.vertices[local_ids].copy()
            X[np.searchsorted(local_ids, vid), comp] += sgn * h
            all_verts.append(X)
            all_cells.append(local_cells + base)
            base += X.shape[0]
            owner += [(k, e) for e in es]
            sign += [sgn] * len(es)
    cells = torch.as_tensor(np.concatenate(all_cells).astype(np.int32), device="cuda")
    verts = torch.as_tensor(np.concatenate(all_verts), device="cuda")
    A = F.tabulate(form, cells, verts).cpu().numpy()
    owner = np.array(owner)
    e_idx = owner[:, 1]
    contrib = np.einsum("ei,eij,ej->e", u[p.dofmap[e_idx]], A, v[p.dofmap[e_idx]])
    fd = np.zeros(len(coords))
    np.add.at(fd, owner[:, 0], contrib * np.array(sign) / (2 * h))
    return fd


def test_adjoint_matches_finite_differences_small(F):
    m = M.unit_cube_tets(3, 0.15, seed=5)
    p = W.make_problem(m, W.POISSON, 2)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(p.n_dof)
    v = rng.standard_normal(p.n_dof)
    _, g, _ = _objective_grad(F, p, u, v)
    coords = [(int(a), int(b)) for a, b in zip(rng.integers(0, m.n_vert, 60), rng.integers(0, 3, 60))]
    fd = _fd_sample(F, p, u, v, coords)
    got = np.array([g[a, b] for a, b in coords])
    assert np.abs(fd - got).max() <= 1e-6 * max(1.0, np.abs(got).max())


def test_adjoint_full_size_p2_poisson(F):
    """56^3 x 6 = 1,053,696 tets, P2 Poisson, u, v iid N(0,1): the GPU gradient at
    1000 seeded vertex coordinates against central differences (h = 1e-6) of the GPU
    forward and against the oracle's shape derivative on the incident cells."""
    p, u, v = W.adjoint_p2(56)
    m = p.mesh
    L, g, _ = _objective_grad(F, p, u, v)
    rng = np.random.default_rng(55)
    vids = rng.choice(m.n_vert, 1000, replace=False)
    coords = [(int(a), int(b)) for a, b in zip(vids, rng.integers(0, 3, 1000))]
    fd = _fd_sample(F, p, u, v, coords)
    got = np.array([g[a, b] for a, b in coords])
    scale = np.abs(got).max()
    assert np.abs(fd - got).max() <= 1e-6 * scale
    # oracle on the cells incident to the first 100 sampled vertices
    sel = np.isin(m.cells, vids[:100]).any(axis=1)
    ref = OS.poisson_shape_gradient(m.vertices, m.cells[sel], 2, p.dofmap[sel], u, v)
    assert np.abs(g[vids[:100]] - ref[vids[:100]]).max() <= 1e-11 * scale
