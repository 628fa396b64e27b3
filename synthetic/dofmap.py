"""Local-to-global degree-of-freedom maps iota(K, .) for continuous Lagrange P_q on the
structured meshes of :mod:`synthetic.mesh` (Section 2.2 of the paper: the maps that
Algorithm 2 uses to add A^K into the global matrix).

The dofmap is an *input* of assembly; this module builds it from mesh topology
only (integer bookkeeping, no arithmetic of the method).

Local dof order on a simplex with local vertices 0..d (the convention the
element tensors use):
  for m = 0, 1, ..., d:
    for every m-dimensional sub-simplex, i.e. vertex subset S of size m+1, taken in
    lexicographic order of S:
      the lattice points k (|k| = q) whose support {j : k_j > 0} is exactly S,
      in descending lexicographic order of k.
So vertices come first (in local vertex order), then edge points (edges 01, 02,
03, 12, 13, 23; the point nearest the lower vertex first), then face points,
then cell-interior points. For P3 on a triangle this puts the bubble last.

Global numbering of scalar dofs: a lattice point with barycentric multi-index k on
cell K sits at integer position P = sum_j k_j * lattice(v_j) of the q-times refined
grid; its global id is the lexicographic index of P in the (q*n+1)^d grid. The id
depends only on the point, so it agrees on every cell sharing the point.

Vector-valued spaces (N-S convection, elasticity) use component-blocked local
numbering i = c*n_s + s and interleaved global numbering g = d*g_s + c.
"""
from __future__ import annotations

import itertools

import numpy as np

from .mesh import SimplexMesh


def local_lattice(d: int, q: int) -> np.ndarray:
    """int64 [n, d+1]: barycentric lattice multi-indices in local dof order."""
    out = []
    for m in range(d + 1):
        for subset in itertools.combinations(range(d + 1), m + 1):
            pts = []
            for k in itertools.product(range(q + 1), repeat=d + 1):
                if sum(k) != q:
                    continue
                support = tuple(j for j in range(d + 1) if k[j] > 0)
                if support == subset:
                    pts.append(k)
            pts.sort(reverse=True)
            out.extend(pts)
    return np.array(out, dtype=np.int64).reshape(-1, d + 1)


def n_local(d: int, q: int) -> int:
    num = 1
    for j in range(1, d + 1):
        num = num * (q + j) // j
    return num


def scalar_dofmap(mesh: SimplexMesh, q: int) -> tuple[np.ndarray, int]:
    """int32 [n_elem, n_s] global ids and the number of global dofs."""
    d = mesh.dim
    lat = local_lattice(d, q)  # [n_s, d+1]
    cell_lat = mesh.lattice[mesh.cells]  # [E, d+1, d]
    pos = np.einsum("sj,ejx->esx", lat, cell_lat)  # [E, n_s, d] in units of h/q
    side = q * mesh.n + 1
    gid = np.zeros(pos.shape[:2], dtype=np.int64)
    for x in range(d):
        gid = gid * side + pos[:, :, x]
    return gid.astype(np.int32), side**d


def vector_dofmap(scalar: np.ndarray, n_dof_scalar: int, d: int) -> tuple[np.ndarray, int]:
    """Component-blocked local order, interleaved global order."""
    E, ns = scalar.shape
    out = np.empty((E, d * ns), dtype=np.int64)
    for c in range(d):
        out[:, c * ns:(c + 1) * ns] = d * scalar.astype(np.int64) + c
    return out.astype(np.int32), d * n_dof_scalar
