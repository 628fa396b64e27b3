"""Named synthetic workloads with the shapes of the paper's test cases (Section 3.3:
mass, Poisson, Navier-Stokes convection, linear elasticity) on seeded structured meshes.

Everything here is input generation: meshes, dofmaps, coefficient vectors and
random fields. Random numbers the method consumes (the convection field w, the
adjoint vectors u, v) are drawn here and passed in as inputs.

Workloads
---------
poisson_p1_tri    unit square, 64x64x2 triangles, jitter 0.2h, seed 1, P1 Poisson
tet_scalar        unit cube, 48^3 x 6 Kuhn tets, jitter 0.15h, seed 2, mass and
                  Poisson with P1..P4
ns_vp2            40^3 x 6 tets, jitter 0.15h, seed 3, vector P2 convection with a
                  global vector-P2 field w, iid N(0,1) per global dof
batched           32 cube meshes, element counts log-uniform in [1e3, 2e5] from
                  seed 4, forms round-robin (elasticity vP1, vP2, vP3, Poisson P2)
adjoint_p2        56^3 x 6 tets, jitter 0.15h, seed 5, P2 Poisson, u, v iid N(0,1)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dofmap import scalar_dofmap, vector_dofmap
from .mesh import SimplexMesh, unit_cube_tets, unit_square_triangles

MASS, POISSON, NS_CONVECTION, ELASTICITY, SOURCE = 0, 1, 2, 3, 4
FORM_NAMES = {MASS: "mass", POISSON: "poisson", NS_CONVECTION: "ns_convection", ELASTICITY: "elasticity",
              SOURCE: "source"}
ELASTICITY_MU = 1.0
ELASTICITY_LAMBDA = 1.25


def is_vector_form(form: int) -> bool:
    return form in (NS_CONVECTION, ELASTICITY)


@dataclass
class FormProblem:
    """One (mesh, form, degree) problem with its dofmap and per-cell coefficients."""

    mesh: SimplexMesh
    form: int
    degree: int
    dofmap: np.ndarray  # int32 [n_elem, n]
    n_dof: int
    coeffs: np.ndarray | None = None  # float64 [n_elem, n_coeff] (N-S: w on each cell)
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return self.mesh.n_elem

    @property
    def n_local(self) -> int:
        return self.dofmap.shape[1]


def make_problem(mesh: SimplexMesh, form: int, degree: int, seed: int = 0) -> FormProblem:
    d = mesh.dim
    sdm, nds = scalar_dofmap(mesh, degree)
    if is_vector_form(form):
        dm, nd = vector_dofmap(sdm, nds, d)
    else:
        dm, nd = sdm, nds
    coeffs = None
    extra = {}
    if form in (NS_CONVECTION, SOURCE):
        rng = np.random.default_rng([seed, 101])
        w = rng.standard_normal(nd)
        coeffs = np.ascontiguousarray(w[dm])
        extra["w_global"] = w
    return FormProblem(mesh, form, degree, dm, nd, coeffs, extra)


def poisson_p1_tri() -> FormProblem:
    return make_problem(unit_square_triangles(64, 0.2, seed=1), POISSON, 1, seed=1)


def tet_scalar_mesh(n: int = 48) -> SimplexMesh:
    return unit_cube_tets(n, 0.15, seed=2)


def ns_vp2(n: int = 40) -> FormProblem:
    return make_problem(unit_cube_tets(n, 0.15, seed=3), NS_CONVECTION, 2, seed=3)


BATCHED_FORMS = [(ELASTICITY, 1), (ELASTICITY, 2), (ELASTICITY, 3), (POISSON, 2)]


def batched_sizes(seed: int = 4, count: int = 32, lo: float = 1e3, hi: float = 2e5) -> list[int]:
    """Cube sizes n_m with 6 n_m^3 close to element counts drawn log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    target = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    return [max(1, int(round((t / 6.0) ** (1.0 / 3.0)))) for t in target]


def batched(seed: int = 4, count: int = 32, scale: float = 1.0) -> list[FormProblem]:
    """The heterogeneous batch: mesh m gets form BATCHED_FORMS[m % 4]."""
    out = []
    for m, n in enumerate(batched_sizes(seed, count)):
        nm = max(1, int(round(n * scale)))
        form, q = BATCHED_FORMS[m % len(BATCHED_FORMS)]
        out.append(make_problem(unit_cube_tets(nm, 0.15, seed=seed * 1000 + m), form, q, seed=seed * 1000 + m))
    return out


def adjoint_p2(n: int = 56) -> tuple[FormProblem, np.ndarray, np.ndarray]:
    prob = make_problem(unit_cube_tets(n, 0.15, seed=5), POISSON, 2, seed=5)
    rng = np.random.default_rng([5, 202])
    u = rng.standard_normal(prob.n_dof)
    v = rng.standard_normal(prob.n_dof)
    return prob, u, v
