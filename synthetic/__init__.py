"""Seeded synthetic inputs (meshes, magnetisations, charges) shared by the
oracle and the CUDA path.  Holds no single-layer-potential arithmetic."""
from . import meshes, fields, workloads  # noqa: F401
