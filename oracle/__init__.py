"""Test infrastructure: a plain, slow, FP64 CPU oracle for element tensors, their
assembly and the shape derivative of u^T A v.

The tensor-representation method (A^K = A0 : G_K, eq. (tensorproduct) of Section 3.2)
is exact: it reproduces the exact integral of the form over each element. The
oracle therefore evaluates the plain definition A^K_{i1 i2} = a_K(phi_i1, phi_i2)
(eq. (elementmatrix), Section 2.2) by quadrature *directly on the physical
element*, without a reference tensor or a geometry tensor:

* ``basis``      Lagrange P_q on a simplex through the barycentric (Silvester)
                 product formula, local dof order as documented there.
* ``quadrature`` Gauss-Legendre nodes by Newton on the Legendre recurrence, and a
                 collapsed (Duffy) rule on the simplex returned in barycentric
                 coordinates.
* ``element``    element tensors of the four test cases of Section 3.3 (mass,
                 Poisson, Navier-Stokes convection, linear elasticity).
* ``assemble``   Algorithm 2 of Section 2.2 into a sorted-column CSR matrix.
* ``shape``      the continuous shape derivative of L = u^T A v for Poisson.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never calls it.
"""
from . import assemble, basis, element, quadrature, shape  # noqa: F401
