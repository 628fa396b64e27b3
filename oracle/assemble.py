"""Assembly of element tensors into a global sparse matrix (oracle).

Algorithm 2 of Section 2.2: A = 0; for each cell K compute A^K, then add it to A
through the local-to-global maps, A[iota(K,i1), iota(K,i2)] += A^K[i1,i2].

``assemble_loop`` is that loop written out over a dict (small meshes only).
``assemble_csr`` computes the same sums with a sort: every (row, col, value)
triple of every element, ordered by (row, col), duplicates summed. The sparsity
pattern is every (row, col) pair that shares a cell, whether or not the summed
value is zero; columns are sorted within each row.
"""
from __future__ import annotations

import numpy as np


def assemble_loop(A_K: np.ndarray, dofmap: np.ndarray) -> dict:
    A = {}
    for e in range(A_K.shape[0]):
        for i1 in range(dofmap.shape[1]):
            for i2 in range(dofmap.shape[1]):
                key = (int(dofmap[e, i1]), int(dofmap[e, i2]))
                A[key] = A.get(key, 0.0) + float(A_K[e, i1, i2])
    return A


def csr_pattern(dofmap: np.ndarray, n_dof: int) -> tuple[np.ndarray, np.ndarray]:
    """Sorted-column CSR pattern (row_ptr int64 [n_dof+1], col int32 [nnz])."""
    E, n = dofmap.shape
    rows = np.repeat(dofmap.astype(np.int64), n, axis=1).reshape(-1)
    cols = np.tile(dofmap.astype(np.int64), (1, n)).reshape(-1)
    key = np.unique(rows * n_dof + cols)
    r = key // n_dof
    c = key % n_dof
    row_ptr = np.zeros(n_dof + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    return np.cumsum(row_ptr), c.astype(np.int32)


def assemble_csr(A_K: np.ndarray, dofmap: np.ndarray, n_dof: int):
    """Global matrix as (row_ptr int64, col int32, val float64)."""
    E, n = dofmap.shape
    rows = np.repeat(dofmap.astype(np.int64), n, axis=1).reshape(-1)
    cols = np.tile(dofmap.astype(np.int64), (1, n)).reshape(-1)
    vals = np.asarray(A_K, dtype=np.float64).reshape(-1)
    key = rows * n_dof + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    start = np.concatenate([[0], np.nonzero(np.diff(key))[0] + 1])
    summed = np.add.reduceat(vals, start)
    ukey = key[start]
    r = ukey // n_dof
    c = (ukey % n_dof).astype(np.int32)
    row_ptr = np.zeros(n_dof + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    return np.cumsum(row_ptr), c, summed


def csr_matvec(row_ptr: np.ndarray, col: np.ndarray, val: np.ndarray, x: np.ndarray) -> np.ndarray:
    rows = np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))
    y = np.zeros(row_ptr.size - 1)
    np.add.at(y, rows, val * x[col])
    return y


def assemble_vector(b_K: np.ndarray, dofmap: np.ndarray, n_dof: int) -> np.ndarray:
    """Algorithm 2 for a linear form: b[iota(K,i)] += b^K[i]."""
    b = np.zeros(n_dof)
    np.add.at(b, dofmap.reshape(-1), np.asarray(b_K, dtype=np.float64).reshape(-1))
    return b
