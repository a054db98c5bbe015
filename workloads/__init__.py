"""Seeded synthetic inputs (meshes, bathymetry, initial states) for tests and benchmarks.

This package is deliberately free of the discretisation's arithmetic; the oracle
and the CUDA path each evaluate these descriptions at their own nodes.
"""
from . import meshes, scenarios  # noqa: F401
