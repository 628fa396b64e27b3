"""ctypes declarations of the C ABI in include/ffc_gb300.h.

Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libffc_gb300.so")

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_u32p = ctypes.POINTER(ctypes.c_uint32)
c_dblp = ctypes.POINTER(ctypes.c_double)
c_vp = ctypes.c_void_p

# name -> (restype, argtypes); every entry point declared in ffc_gb300.h
SIGNATURES = {
    "ffc_form_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(c_vp)]),
    "ffc_form_info": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "ffc_form_rank": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int)]),
    "ffc_form_reference_tensor": (ctypes.c_int, [c_vp, c_vp]),
    "ffc_form_set_algorithm": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "ffc_form_destroy": (None, [c_vp]),
    "ffc_tabulate": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int,
                                    c_vp]),
    "ffc_csr_pattern": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, c_vp, ctypes.c_int64, c_vp, c_i64p, c_vp,
                                       ctypes.c_int64, c_vp]),
    "ffc_assemble": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, c_vp,
                                    ctypes.c_int64, ctypes.c_int, c_vp]),
    "ffc_assemble_pair": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, c_vp,
                                         ctypes.c_int64, ctypes.c_int, c_vp]),
    "ffc_scatter_add": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, c_vp, ctypes.c_int, c_vp, c_vp, ctypes.c_int64,
                                       c_vp]),
    "ffc_tabulate_adjoint": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, c_vp]),
    "ffc_tabulate_static": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp,
                                           ctypes.c_int, c_vp, c_u32p]),
    "ffc_batch_create": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_vp)]),
    "ffc_batch_tune": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "ffc_batch_run": (ctypes.c_int, [c_vp, ctypes.c_int, c_vp]),
    "ffc_batch_info": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "ffc_batch_destroy": (None, [c_vp]),
    "ffc_row_plan_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, c_vp, ctypes.c_int64, c_vp, c_vp,
                                           ctypes.c_int64, c_vp, ctypes.POINTER(c_vp)]),
    "ffc_row_plan_info": (ctypes.c_int, [c_vp, c_i64p, c_i64p, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "ffc_row_plan_layout": (ctypes.c_int, [c_vp, c_i64p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), c_i64p]),
    "ffc_row_plan_destroy": (None, [c_vp]),
    "ffc_assemble_rows_pair": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int,
                                              c_vp]),
    "ffc_assemble_rows": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.c_int64, c_vp, ctypes.c_int, c_vp]),
    "ffc_qform_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(c_vp)]),
    "ffc_qform_info": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "ffc_qform_reference_tensor": (ctypes.c_int, [c_vp, c_vp]),
    "ffc_qform_rule": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "ffc_qform_destroy": (None, [c_vp]),
    "ffc_tabulate_quadrature": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, ctypes.c_int,
                                               c_vp]),
    "ffc_assemble_quadrature": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp,
                                               ctypes.c_int64, ctypes.c_int, c_vp]),
    "ffc_diag_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, c_vp]),
    "ffc_diag_peak": (ctypes.c_int, [ctypes.c_int, c_dblp, c_dblp, c_vp]),
    "ffc_status_poll": (ctypes.c_int, [c_vp, c_u32p]),
    "ffc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ffc_last_error": (ctypes.c_char_p, []),
}

class BatchItem(ctypes.Structure):
    """ffc_batch_item."""

    _fields_ = [("form", c_vp), ("n_elem", ctypes.c_int64), ("cells", c_vp), ("vertices", c_vp),
                ("n_vert", ctypes.c_int64), ("coeffs", c_vp), ("slot", c_vp), ("csr_val", c_vp),
                ("nnz", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_1112_0402_gb300.build.build() "
                "(nvcc, sm_103a). There is no CPU fallback.")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib
