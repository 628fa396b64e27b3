"""ffc_tabulate_static: the entry point for callers that cannot allocate device memory
(its reference tensor and status word sit in a fixed device array inside the library).
Called through the C ABI and compared with ffc_tabulate on two calls in a row; this
file is collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-6


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).double()
    b = b.reshape(b.shape[0], -1).double()
    return ((a - b).norm(dim=1) / b.norm(dim=1)).max().item()


def _static_call(L, form, cells, verts, coeffs, out, precision):
    import torch

    flags = ctypes.c_uint32(99)
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    rc = L.ffc_tabulate_static(form.handle, cells.shape[0], vp(cells), vp(verts), verts.shape[0], vp(coeffs),
                               vp(out), precision, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               ctypes.byref(flags))
    return rc, flags.value


def test_static_scratch_entry_point_matches_ffc_tabulate():
    import torch

    from paper_1112_0402_gb300 import _capi
    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    L = _capi.lib()
    cases = [(W.POISSON, 3, F.FP64, FP64_TOL, None), (W.NS_CONVECTION, 2, F.FP32, FP32_TOL, 3)]
    for kind, q, prec, tol, seed in cases:
        m = M.unit_cube_tets(3, 0.15, seed=4)
        p = W.make_problem(m, kind, q, seed=seed or 0)
        form = F.Form(kind, F.TETRAHEDRON, q)
        cells = torch.as_tensor(m.cells, device="cuda")
        verts = torch.as_tensor(m.vertices, device="cuda")
        coeffs = torch.as_tensor(p.coeffs, device="cuda") if p.coeffs is not None else None
        ref = F.tabulate(form, cells, verts, coeffs=coeffs, precision=prec)
        dt = torch.float64 if prec == F.FP64 else torch.float32
        out = torch.full_like(ref, float("nan"), dtype=dt)
        rc, flags = _static_call(L, form, cells, verts, coeffs, out, prec)
        assert rc == 0, L.ffc_last_error().decode()
        assert flags == 0
        assert _rel(out, ref) <= tol
    # a form whose reference tensor does not fit the fixed array is refused up front
    big = F.Form(W.ELASTICITY, F.TETRAHEDRON, 3)
    m = M.unit_cube_tets(1)
    cells = torch.as_tensor(m.cells, device="cuda")
    verts = torch.as_tensor(m.vertices, device="cuda")
    out = torch.empty((6, 60, 60), dtype=torch.float64, device="cuda")
    rc, _ = _static_call(L, big, cells, verts, None, out, F.FP64)
    assert rc == -1
    assert np.isfinite(ref.cpu().numpy()).all()


def test_static_entry_point_through_the_python_binding():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    m = M.unit_cube_tets(3, 0.15, seed=6)
    form = F.Form(W.MASS, F.TETRAHEDRON, 2)
    cells = torch.as_tensor(m.cells, device="cuda")
    verts = torch.as_tensor(m.vertices, device="cuda")
    ref = F.tabulate(form, cells, verts, precision="fp32")
    for _ in range(2):  # two calls in a row reuse the fixed array
        out, flags = F.tabulate_static(form, cells, verts, precision="fp32")
        assert flags == 0
        assert torch.equal(out, ref)
