"""Seeded structured simplex meshes (triangles on the unit square, Kuhn tetrahedra on
the unit cube) with jittered interior vertices.

This module only builds inputs: vertex coordinates, cell-to-vertex tables and the
integer lattice coordinates that identify each vertex. It holds no arithmetic of the
tensor-representation method. The affine simplices it produces are the element
families the method is stated for (Section 3.2 of the paper assumes affine maps
from a reference simplex; Section 5.3 lists Lagrange elements on triangles and
tetrahedra).

Conventions
-----------
* Vertex id is lexicographic in the grid index, the first axis varying slowest:
  ``id = i*(n+1) + j`` (2-D) and ``id = (i*(n+1) + j)*(n+1) + k`` (3-D).
* Triangles: grid cell (i, j) is cut along its (i,j)-(i+1,j+1) diagonal into
  ``[(i,j), (i+1,j), (i+1,j+1)]`` and ``[(i,j), (i+1,j+1), (i,j+1)]``.
* Tetrahedra: each hex is cut into the 6 Kuhn (Freudenthal) tetrahedra around its
  (0,0,0)-(1,1,1) diagonal, one per permutation of the axes; the tetrahedron for
  permutation p has vertices c, c+e_p0, c+e_p0+e_p1, c+(1,1,1). The mesh is
  conforming. Half of the tetrahedra have negative orientation; vertex order is
  kept as built.
* Jitter moves interior vertices only, each coordinate independently uniform in
  [-a*h, a*h], drawn with ``numpy.random.default_rng(seed)`` (PCG64). Boundary
  vertices stay on the boundary, so the domain measure stays exactly 1.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class SimplexMesh:
    """A structured simplex mesh.

    vertices : float64 [n_v, d]  physical coordinates
    cells    : int32   [n_elem, d+1] vertex ids, local vertex order as built
    lattice  : int64   [n_v, d]  integer grid coordinates (vertex = lattice * h before jitter)
    n        : cells per axis
    """

    vertices: np.ndarray
    cells: np.ndarray
    lattice: np.ndarray
    n: int

    @property
    def dim(self) -> int:
        return self.vertices.shape[1]

    @property
    def n_elem(self) -> int:
        return self.cells.shape[0]

    @property
    def n_vert(self) -> int:
        return self.vertices.shape[0]


def _grid_lattice(n: int, d: int) -> np.ndarray:
    axes = [np.arange(n + 1, dtype=np.int64)] * d
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def _jitter(lattice: np.ndarray, n: int, jitter: float, seed: int) -> np.ndarray:
    h = 1.0 / n
    x = lattice.astype(np.float64) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        interior = np.all((lattice > 0) & (lattice < n), axis=1)
        disp = rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), lattice.shape[1]))
        x[interior] += disp
    return x


def unit_square_triangles(n: int, jitter: float = 0.0, seed: int = 0) -> SimplexMesh:
    """2*n*n triangles on [0,1]^2."""
    lat = _grid_lattice(n, 2)
    vid = lambda i, j: i * (n + 1) + j  # noqa: E731
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.reshape(-1)
    j = j.reshape(-1)
    t0 = np.stack([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)], axis=1)
    t1 = np.stack([vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)], axis=1)
    cells = np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int32)
    return SimplexMesh(_jitter(lat, n, jitter, seed), cells, lat, n)


KUHN_PERMUTATIONS = list(itertools.permutations(range(3)))


def unit_cube_tets(n: int, jitter: float = 0.0, seed: int = 0) -> SimplexMesh:
    """6*n^3 Kuhn tetrahedra on [0,1]^3."""
    lat = _grid_lattice(n, 3)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    corner = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1)
    eye = np.eye(3, dtype=np.int64)

    def vid(c):
        return (c[:, 0] * (n + 1) + c[:, 1]) * (n + 1) + c[:, 2]

    tets = []
    for p in KUHN_PERMUTATIONS:
        c1 = corner + eye[p[0]]
        c2 = c1 + eye[p[1]]
        c3 = c2 + eye[p[2]]
        tets.append(np.stack([vid(corner), vid(c1), vid(c2), vid(c3)], axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return SimplexMesh(_jitter(lat, n, jitter, seed), cells, lat, n)


def gather_cell_vertices(mesh: SimplexMesh) -> np.ndarray:
    """float64 [n_elem, d+1, d]: the coordinates of each cell's vertices in local order."""
    return mesh.vertices[mesh.cells]
