"""GB300 (sm_103a) tensor representation of variational forms: batched element
tensors A^K = A0 : G_K and their fused insertion into a global CSR matrix
(Kirby & Logg, "A Compiler for Variational Forms", Sections 2.2 and 3.2).

The compute path is the C-ABI library ``libffc_gb300.so`` (include/ffc_gb300.h);
this package only marshals arguments to it.
"""
from .api import (ALG_AUTO, ALG_BLOCK, ALG_DENSE, BF16X3, ELASTICITY, FLAG_BOUNDS, FLAG_DEGENERATE, FLAG_TIMEOUT, FP32, FP64, FP64_OZAKI, MASS, NS_CONVECTION, PEAKS, PRECISIONS,  # noqa
                  POISSON, SOURCE, TETRAHEDRON, TF32, TF32X3, TRIANGLE, Batch, FFCError, Form, QForm, RowPlan, assemble,
                  assemble_pair, assemble_quadrature, assemble_rows, assemble_rows_pair, csr_pattern, diag_bounded_wait, diag_peak,
                  scatter_add, status_poll, tabulate, tabulate_adjoint, tabulate_quadrature, tabulate_static)
