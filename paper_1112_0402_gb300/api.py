"""Python binding of the C ABI (argument marshalling only: every step runs in the
library's CUDA kernels). PyTorch provides device memory and streams.

    form = Form(POISSON, TETRAHEDRON, 2)
    A_K = tabulate(form, cells, vertices)                 # [n_elem, n, n] on the GPU
    row_ptr, col, slot = csr_pattern(dofmap, n_dof)       # host, setup
    assemble(form, cells, vertices, slot_dev, csr_val)    # csr_val[slot] += A^K
    plan = RowPlan(dofmap_dev, n_dof, row_ptr_dev, col_dev)  # mass / Poisson, once per mesh
    assemble_rows(form, plan, cells, vertices, csr_val)   # csr_val = A (row-owner, fixed-point sums)

A linear form (SOURCE, rank 1) has element vectors [n_elem, n]; its assembly adds
them into a global vector, with the dof map in place of the slots:

    L = Form(SOURCE, TETRAHEDRON, 2)
    b = torch.zeros(n_dof, dtype=torch.float64, device="cuda")
    assemble(L, cells, vertices, dofmap_dev, b, coeffs=f_on_cells)
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._capi import lib

MASS, POISSON, NS_CONVECTION, ELASTICITY, SOURCE = 0, 1, 2, 3, 4
TRIANGLE, TETRAHEDRON = 2, 3
FP64, FP32, TF32, TF32X3, BF16X3, FP64_OZAKI = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "tf32x3": TF32X3, "bf16x3": BF16X3,
              "fp64_ozaki": FP64_OZAKI}
FLAG_DEGENERATE, FLAG_BOUNDS, FLAG_TIMEOUT = 1, 2, 4
ALG_AUTO, ALG_DENSE, ALG_BLOCK = 0, 1, 2


class FFCError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        msg = L.ffc_status_string(code).decode()
        detail = L.ffc_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))
        self.code = code


def _check(code: int, where: str) -> None:
    if code != 0:
        raise FFCError(code, where)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, name, shape=None):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Form:
    """A compiled form: the reference tensor A0 of (kind, cell, degree)."""

    def __init__(self, kind: int, cell: int, degree: int, mu: float = 1.0, lmbda: float = 1.25,
                 algorithm: int = ALG_AUTO):
        h = ctypes.c_void_p()
        _check(lib().ffc_form_create(kind, cell, degree, mu, lmbda, ctypes.byref(h)), "ffc_form_create")
        self._h = h
        _check(lib().ffc_form_set_algorithm(h, algorithm), "ffc_form_set_algorithm")
        self.kind, self.cell, self.degree = kind, cell, degree
        n, na, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ffc_form_info(h, ctypes.byref(n), ctypes.byref(na), ctypes.byref(nc)), "ffc_form_info")
        self.n_local, self.n_alpha, self.n_coeff = n.value, na.value, nc.value
        r = ctypes.c_int()
        _check(lib().ffc_form_rank(h, ctypes.byref(r)), "ffc_form_rank")
        self.rank = r.value

    @property
    def tensor_shape(self) -> tuple:
        """Shape of one element tensor: (n, n), or (n,) for a linear form."""
        return (self.n_local,) * self.rank

    @property
    def handle(self):
        return self._h

    @property
    def dim(self) -> int:
        return self.cell

    def reference_tensor(self) -> np.ndarray:
        out = np.empty((self.n_local ** self.rank, self.n_alpha), dtype=np.float64)
        _check(lib().ffc_form_reference_tensor(self._h, out.ctypes.data_as(ctypes.c_void_p)),
               "ffc_form_reference_tensor")
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ffc_form_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tabulate(form: Form, cells, vertices, coeffs=None, precision="fp64", out=None, stream=None):
    """Element tensors [n_elem, n, n] ([n_elem, n] for a linear form; float64 for fp64,
    float32 otherwise)."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    shp = (n_elem,) + form.tensor_shape
    dt = torch.float64 if p == FP64 else torch.float32
    if out is None:
        out = torch.empty(shp, dtype=dt, device=vertices.device)
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    w = _dev_ptr(coeffs, torch.float64, "coeffs", (n_elem, form.n_coeff)) if form.n_coeff else None
    o = _dev_ptr(out, dt, "out", shp)
    _check(lib().ffc_tabulate(form.handle, n_elem, c, v, vertices.shape[0], w, o, p, _stream(stream)),
           "ffc_tabulate")
    return out


def tabulate_static(form: Form, cells, vertices, coeffs=None, precision="fp64", out=None, stream=None):
    """tabulate() through the allocation-free entry point (ffc_tabulate_static): the
    reference tensor is staged in a fixed device array compiled into the library.
    FP64 or FP32 only; synchronises ``stream`` and returns (A_K, device status bits)."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    shp = (n_elem,) + form.tensor_shape
    dt = torch.float64 if p == FP64 else torch.float32
    if out is None:
        out = torch.empty(shp, dtype=dt, device=vertices.device)
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    w = _dev_ptr(coeffs, torch.float64, "coeffs", (n_elem, form.n_coeff)) if form.n_coeff else None
    o = _dev_ptr(out, dt, "out", shp)
    flags = ctypes.c_uint32()
    _check(lib().ffc_tabulate_static(form.handle, n_elem, c, v, vertices.shape[0], w, o, p, _stream(stream),
                                     ctypes.byref(flags)), "ffc_tabulate_static")
    return out, flags.value


def csr_pattern(dofmap: np.ndarray, n_dof: int, with_slots: bool = True):
    """Sorted-column CSR pattern (row_ptr int64, col int32) and slots int32 [n_elem, n, n]."""
    dm = np.ascontiguousarray(dofmap, dtype=np.int32)
    n_elem, n = dm.shape
    row_ptr = np.empty(n_dof + 1, dtype=np.int64)
    nnz = ctypes.c_int64()
    L = lib()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(L.ffc_csr_pattern(n_elem, n, vp(dm), n_dof, vp(row_ptr), ctypes.byref(nnz), None, 0, None),
           "ffc_csr_pattern")
    col = np.empty(nnz.value, dtype=np.int32)
    slot = np.empty((n_elem, n, n), dtype=np.int32) if with_slots else None
    _check(L.ffc_csr_pattern(n_elem, n, vp(dm), n_dof, vp(row_ptr), ctypes.byref(nnz), vp(col), col.size,
                             vp(slot) if slot is not None else None), "ffc_csr_pattern")
    return row_ptr, col, slot


def assemble(form: Form, cells, vertices, slot, csr_val, coeffs=None, precision="fp64", stream=None):
    """csr_val[slot[e, i1, i2]] += A^K[e, i1, i2] for all cells (accumulates). For a
    linear form ``slot`` is the dof map [n_elem, n] and ``csr_val`` the global vector."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    w = _dev_ptr(coeffs, torch.float64, "coeffs", (n_elem, form.n_coeff)) if form.n_coeff else None
    s = _dev_ptr(slot, torch.int32, "slot", (n_elem,) + form.tensor_shape)
    val = _dev_ptr(csr_val, torch.float64, "csr_val")
    _check(lib().ffc_assemble(form.handle, n_elem, c, v, vertices.shape[0], w, s, val, csr_val.numel(), p,
                              _stream(stream)), "ffc_assemble")
    return csr_val


class RowPlan:
    """Row view of a dof map and its CSR pattern for :func:`assemble_rows`
    (ffc_row_plan_create; built on the device, synchronises the stream).

    dofmap int32 [n_elem, n_local], row_ptr int64 [n_dof + 1] and col int32 [nnz] are
    CUDA tensors (the pattern of :func:`csr_pattern`); they may be freed afterwards."""

    def __init__(self, dofmap, n_dof: int, row_ptr, col, stream=None):
        import torch

        n_elem, n_local = dofmap.shape
        d = _dev_ptr(dofmap, torch.int32, "dofmap")
        rp = _dev_ptr(row_ptr, torch.int64, "row_ptr", (n_dof + 1,))
        c = _dev_ptr(col, torch.int32, "col")
        h = ctypes.c_void_p()
        _check(lib().ffc_row_plan_create(n_elem, n_local, d, n_dof, rp, c, col.numel(), _stream(stream),
                                         ctypes.byref(h)), "ffc_row_plan_create")
        self._h = h
        self.n_local = n_local
        nd, nnz, mr, mi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ffc_row_plan_info(h, ctypes.byref(nd), ctypes.byref(nnz), ctypes.byref(mr), ctypes.byref(mi)),
               "ffc_row_plan_info")
        self.n_dof, self.nnz, self.max_row, self.max_incidence = nd.value, nnz.value, mr.value, mi.value
        nc, vm, pm, gr, nb = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().ffc_row_plan_layout(h, ctypes.byref(nc), ctypes.byref(vm), ctypes.byref(pm), ctypes.byref(gr),
                                         ctypes.byref(nb)), "ffc_row_plan_layout")
        self.n_chunks, self.max_chunk_values, self.max_chunk_pairs = nc.value, vm.value, pm.value
        self.max_region_bytes, self.device_bytes = gr.value, nb.value

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ffc_row_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assemble_rows(form: Form, plan: RowPlan, cells, vertices, csr_val, precision="fp32", stream=None):
    """csr_val = the assembled matrix of a mass or Poisson form (overwritten, no zeroing
    needed), by row-owner assembly with exact fixed-point sums (ffc_assemble_rows)."""
    import torch

    p = _prec(precision)
    c = _dev_ptr(cells, torch.int32, "cells", (cells.shape[0], form.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    val = _dev_ptr(csr_val, torch.float64, "csr_val", (plan.nnz,))
    _check(lib().ffc_assemble_rows(form.handle, plan.handle, c, v, vertices.shape[0], val, p, _stream(stream)),
           "ffc_assemble_rows")
    return csr_val


def assemble_rows_pair(form_a: Form, form_b: Form, plan: RowPlan, cells, vertices, csr_val_a, csr_val_b,
                       precision="fp32", stream=None):
    """Two forms on the plan's space into two matrices (overwritten) by row-owner assembly
    (ffc_assemble_rows_pair); the (mass, Poisson) pair is one pass."""
    import torch

    p = _prec(precision)
    c = _dev_ptr(cells, torch.int32, "cells", (cells.shape[0], form_a.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    va = _dev_ptr(csr_val_a, torch.float64, "csr_val_a", (plan.nnz,))
    vb = _dev_ptr(csr_val_b, torch.float64, "csr_val_b", (plan.nnz,))
    _check(lib().ffc_assemble_rows_pair(form_a.handle, form_b.handle, plan.handle, c, v, vertices.shape[0], va, vb, p,
                                        _stream(stream)), "ffc_assemble_rows_pair")
    return csr_val_a, csr_val_b


def assemble_pair(form_a: Form, form_b: Form, cells, vertices, slot, csr_val_a, csr_val_b, precision="fp32",
                  stream=None):
    """Two forms on one space into two matrices sharing the pattern (ffc_assemble_pair):
    csr_val_a[slot] += A_a^K, csr_val_b[slot] += A_b^K. The (mass, Poisson) pair in FP32 is
    one launch (geometry and slot loads shared)."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form_a.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    s = _dev_ptr(slot, torch.int32, "slot", (n_elem,) + form_a.tensor_shape)
    va = _dev_ptr(csr_val_a, torch.float64, "csr_val_a")
    vb = _dev_ptr(csr_val_b, torch.float64, "csr_val_b", tuple(csr_val_a.shape))
    _check(lib().ffc_assemble_pair(form_a.handle, form_b.handle, n_elem, c, v, vertices.shape[0], s, va, vb,
                                   csr_val_a.numel(), p, _stream(stream)), "ffc_assemble_pair")
    return csr_val_a, csr_val_b


class QForm:
    """A mass or Poisson form in the quadrature representation (Section 3.4): A~0 with a
    quadrature-point index, for cells mapped by a geometry interpolant of degree
    `geometry_degree` (2: curved, isoparametric-style cells)."""

    def __init__(self, kind: int, cell: int, degree: int, geometry_degree: int = 2, quad_degree: int | None = None):
        d = 2 if cell == TRIANGLE else 3
        if quad_degree is None:  # the mass integrand's degree on a map of this degree
            quad_degree = 2 * degree + d * (geometry_degree - 1)
        h = ctypes.c_void_p()
        _check(lib().ffc_qform_create(kind, cell, degree, geometry_degree, quad_degree, ctypes.byref(h)),
               "ffc_qform_create")
        self._h = h
        self.kind, self.cell, self.degree, self.dim = kind, cell, degree, d
        self.geometry_degree, self.quad_degree = geometry_degree, quad_degree
        n, g, nq, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ffc_qform_info(h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(nq), ctypes.byref(k)),
               "ffc_qform_info")
        self.n_local, self.n_geometry, self.n_points, self.k_contract = n.value, g.value, nq.value, k.value

    @property
    def handle(self):
        return self._h

    def reference_tensor(self) -> np.ndarray:
        out = np.empty((self.n_local ** 2, self.k_contract), dtype=np.float64)
        _check(lib().ffc_qform_reference_tensor(self._h, out.ctypes.data_as(ctypes.c_void_p)),
               "ffc_qform_reference_tensor")
        return out

    def rule(self) -> tuple[np.ndarray, np.ndarray]:
        X = np.empty((self.n_points, self.dim), dtype=np.float64)
        w = np.empty(self.n_points, dtype=np.float64)
        _check(lib().ffc_qform_rule(self._h, X.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)),
               "ffc_qform_rule")
        return X, w

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ffc_qform_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tabulate_quadrature(form: QForm, cells, nodes, precision="fp64", out=None, stream=None):
    """Element tensors of curved cells by quadrature as a contraction (ffc_tabulate_quadrature).
    cells int32 [n_elem, n_geometry] geometry node ids, nodes float64 [n_nodes, d]."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.n_geometry))
    v = _dev_ptr(nodes, torch.float64, "nodes", (nodes.shape[0], form.dim))
    dt = torch.float64 if p in (FP64, FP64_OZAKI) else torch.float32
    if out is None:
        out = torch.empty((n_elem, form.n_local, form.n_local), dtype=dt, device=cells.device)
    o = _dev_ptr(out, dt, "out", (n_elem, form.n_local, form.n_local))
    _check(lib().ffc_tabulate_quadrature(form.handle, n_elem, c, v, nodes.shape[0], o, p, _stream(stream)),
           "ffc_tabulate_quadrature")
    return out


def assemble_quadrature(form: QForm, cells, nodes, slot, csr_val, precision="fp64", stream=None):
    """csr_val[slot] += A_K of curved cells (ffc_assemble_quadrature)."""
    import torch

    p = _prec(precision)
    n_elem = cells.shape[0]
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.n_geometry))
    v = _dev_ptr(nodes, torch.float64, "nodes", (nodes.shape[0], form.dim))
    s = _dev_ptr(slot, torch.int32, "slot", (n_elem, form.n_local, form.n_local))
    val = _dev_ptr(csr_val, torch.float64, "csr_val")
    _check(lib().ffc_assemble_quadrature(form.handle, n_elem, c, v, nodes.shape[0], s, val, csr_val.numel(), p,
                                         _stream(stream)), "ffc_assemble_quadrature")
    return csr_val


def scatter_add(A_K, slot, csr_val, stream=None):
    """The insertion step alone: csr_val[slot[e, ...]] += A_K[e, ...] (FP64 atomics).
    A_K float64 or float32 [n_elem, ...]; slot int32 of the same shape."""
    import torch

    if A_K.dtype not in (torch.float64, torch.float32):
        raise TypeError("A_K must be float64 or float32")
    n_elem = A_K.shape[0]
    n_entries = int(np.prod(A_K.shape[1:])) if A_K.dim() > 1 else 1
    a = _dev_ptr(A_K, A_K.dtype, "A_K")
    s = _dev_ptr(slot, torch.int32, "slot", tuple(A_K.shape))
    val = _dev_ptr(csr_val, torch.float64, "csr_val")
    p = FP64 if A_K.dtype == torch.float64 else FP32
    _check(lib().ffc_scatter_add(n_elem, n_entries, a, p, s, val, csr_val.numel(), _stream(stream)),
           "ffc_scatter_add")
    return csr_val


def tabulate_adjoint(form: Form, cells, vertices, dA_K, dvertices=None, stream=None):
    """dL/dvertices (accumulated into ``dvertices``) for the upstream gradient dA_K."""
    import torch

    n_elem = cells.shape[0]
    n = form.n_local
    if dvertices is None:
        dvertices = torch.zeros_like(vertices)
    c = _dev_ptr(cells, torch.int32, "cells", (n_elem, form.dim + 1))
    v = _dev_ptr(vertices, torch.float64, "vertices")
    g = _dev_ptr(dA_K, torch.float64, "dA_K", (n_elem, n, n))
    dv = _dev_ptr(dvertices, torch.float64, "dvertices", tuple(vertices.shape))
    _check(lib().ffc_tabulate_adjoint(form.handle, n_elem, c, v, vertices.shape[0], g, dv, _stream(stream)),
           "ffc_tabulate_adjoint")
    return dvertices


def diag_bounded_wait(polls: int = 4096, stream=None) -> None:
    """Launches the failure-detection probe (ffc_diag_bounded_wait): a bounded device
    wait that nothing ends; status_poll() then reports FLAG_TIMEOUT."""
    _check(lib().ffc_diag_bounded_wait(polls, _stream(stream)), "ffc_diag_bounded_wait")


PEAKS = {"fp64_fma": 0, "fp32_fma": 1, "tf32_mma": 2, "bf16_mma": 3, "smem_atomic_u32": 4}


def diag_peak(kind: str, stream=None) -> tuple[float, float]:
    """Measured compute ceiling of the current device (ffc_diag_peak): (operations per
    second, seconds of the timed launch). kind is one of PEAKS."""
    rate, sec = ctypes.c_double(), ctypes.c_double()
    _check(lib().ffc_diag_peak(PEAKS[kind], ctypes.byref(rate), ctypes.byref(sec), _stream(stream)),
           "ffc_diag_peak")
    return rate.value, sec.value


def status_poll(stream=None) -> int:
    flags = ctypes.c_uint32()
    _check(lib().ffc_status_poll(_stream(stream), ctypes.byref(flags)), "ffc_status_poll")
    return flags.value


class Batch:
    """Many assembly problems in one persistent launch (ffc_batch_*).

    items: sequence of dicts with keys form, cells, vertices, slot, csr_val
    (device tensors as for :func:`assemble`); the arithmetic is FP32 contraction with
    FP64 CSR accumulation."""

    def __init__(self, items, zero_csr: bool = True):
        import torch

        from ._capi import BatchItem

        arr = (BatchItem * len(items))()
        self._keep = []
        for k, it in enumerate(items):
            f = it["form"]
            n = f.n_local
            cells, verts, slot, val = it["cells"], it["vertices"], it["slot"], it["csr_val"]
            ne = cells.shape[0]
            arr[k].form = f.handle
            arr[k].n_elem = ne
            arr[k].cells = _dev_ptr(cells, torch.int32, "cells", (ne, f.dim + 1))
            arr[k].vertices = _dev_ptr(verts, torch.float64, "vertices")
            arr[k].n_vert = verts.shape[0]
            arr[k].coeffs = None
            arr[k].slot = _dev_ptr(slot, torch.int32, "slot", (ne, n, n))
            arr[k].csr_val = _dev_ptr(val, torch.float64, "csr_val")
            arr[k].nnz = val.numel()
            self._keep.append((f, cells, verts, slot, val))
        h = ctypes.c_void_p()
        _check(lib().ffc_batch_create(arr, len(items), int(zero_csr), ctypes.byref(h)), "ffc_batch_create")
        self._h = h

    def tune(self, stream=None) -> int:
        """Picks the fastest tile variant; returns its cells per thread group and tile."""
        c, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().ffc_batch_tune(self._h, _stream(stream), ctypes.byref(c), ctypes.byref(b)), "ffc_batch_tune")
        self.threads_per_block = b.value
        return c.value

    def run(self, graph: bool = False, stream=None) -> None:
        _check(lib().ffc_batch_run(self._h, int(graph), _stream(stream)), "ffc_batch_run")

    def info(self):
        n, tiles, ke, blk = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ffc_batch_info(self._h, ctypes.byref(n), ctypes.byref(tiles), ctypes.byref(ke),
                                    ctypes.byref(blk)), "ffc_batch_info")
        return {"items": n.value, "tiles": tiles.value, "cells_per_tile_group": ke.value,
                "threads_per_block": blk.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ffc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
