"""Seeded synthetic inputs (meshes and analytic flow fields) shared by the
oracle tests, the CUDA-path tests and the benchmark.  Holds no SD arithmetic."""
from . import fields, meshes  # noqa: F401
from .workloads import WORKLOADS, build_workload  # noqa: F401
