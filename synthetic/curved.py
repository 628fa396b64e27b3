"""Curved (quadratic-geometry) simplex meshes: the inputs of the quadrature
representation on non-affine cells (Section 3.4, "Curvilinear elements").

The P2 lattice nodes of the structured meshes of :mod:`synthetic.mesh` (vertices and
edge midpoints of the straight cells, numbered like the P2 dofs of
:func:`synthetic.dofmap.scalar_dofmap`) are moved by a smooth deformation that vanishes
on the boundary of the unit square or cube,

    x -> x + eps * prod_a sin(pi x_a) * v,   v a fixed direction,

so every interior cell becomes a quadratic-geometry cell with curved edges while the
domain stays the unit square / cube. Node ids, lattice positions and one smooth input
field only; none of the method's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .dofmap import scalar_dofmap
from .mesh import SimplexMesh, unit_cube_tets, unit_square_triangles


@dataclass
class CurvedMesh:
    mesh: SimplexMesh   # the straight mesh (topology of the P_q dof maps)
    cells: np.ndarray   # int32 [n_elem, n_g]: geometry node ids, P2 local order
    nodes: np.ndarray   # float64 [n_nodes, d]: node coordinates

    @property
    def dim(self) -> int:
        return self.nodes.shape[1]

    @property
    def n_elem(self) -> int:
        return self.cells.shape[0]


def curved_mesh(d: int, n: int, eps: float = 0.08, seed: int = 7) -> CurvedMesh:
    mesh = unit_square_triangles(n, 0.0, seed) if d == 2 else unit_cube_tets(n, 0.0, seed)
    cells, n_nodes = scalar_dofmap(mesh, 2)
    side = 2 * n + 1
    idx = np.arange(n_nodes, dtype=np.int64)
    pos = np.empty((n_nodes, d), dtype=np.int64)
    for a in range(d - 1, -1, -1):  # ids are lexicographic, first coordinate slowest
        pos[:, a] = idx % side
        idx = idx // side
    x = pos.astype(np.float64) / (2 * n)
    direction = np.array([1.0, 0.6, -0.8][:d])
    bump = np.prod(np.sin(np.pi * x), axis=1)
    nodes = x + eps * bump[:, None] * direction[None, :]
    return CurvedMesh(mesh, cells.astype(np.int32), nodes)


def gather_nodes(cm: CurvedMesh) -> np.ndarray:
    """[n_elem, n_g, d] node coordinates of every cell."""
    return cm.nodes[cm.cells]
