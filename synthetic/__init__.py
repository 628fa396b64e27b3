"""Seeded synthetic inputs (meshes, dofmaps, coefficient fields) shared by the tests,
the benchmark and the oracle checks. No arithmetic of the method lives here."""
from . import dofmap, mesh, workloads  # noqa: F401
