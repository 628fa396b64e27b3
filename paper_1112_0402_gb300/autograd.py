"""torch.autograd.Function over ffc_tabulate (forward) and ffc_tabulate_adjoint
(backward): element tensors of the Poisson form as a differentiable function of the
vertex coordinates (shape derivatives). FP64 in both directions."""
from __future__ import annotations

import torch

from . import api


class _ElementTensors(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vertices, form, cells):
        A = api.tabulate(form, cells, vertices, precision=api.FP64)
        ctx.save_for_backward(vertices, cells)
        ctx.form = form
        return A

    @staticmethod
    def backward(ctx, grad):
        vertices, cells = ctx.saved_tensors
        dv = api.tabulate_adjoint(ctx.form, cells, vertices, grad.contiguous().to(torch.float64))
        return dv, None, None


def element_tensors(form: api.Form, cells: torch.Tensor, vertices: torch.Tensor) -> torch.Tensor:
    """A_K [n_elem, n, n] (float64), differentiable with respect to ``vertices``."""
    if form.kind != api.POISSON:
        raise NotImplementedError("the adjoint is built for the Poisson form")
    return _ElementTensors.apply(vertices, form, cells)
