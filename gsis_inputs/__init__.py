"""Seeded synthetic inputs shared by the solver's tests, the benchmark and the oracle.

This package generates meshes, quadrature grids, per-cell macroscopic states and
distribution functions.  It holds none of the GSIS method's arithmetic.
"""
from . import fields, mesh, quadrature, workloads  # noqa: F401
