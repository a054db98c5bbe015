"""GB300-native nodal DG shallow-water engine (arXiv:1403.1661): Python binding.

The numerical work is done by the CUDA kernels of libswe_gb300.so behind the C
ABI in include/swe.h; this package only marshals arguments and provides device
memory and streams through PyTorch.
"""
from . import _native  # noqa: F401
from .batch import Batch, apply_tuning, tune  # noqa: F401
from .solver import (Mesh, Solver, ref_nodes, ref_operator, ref_sizes,  # noqa: F401
                     scenario_inputs, solver_from_scenario)

__all__ = ["Batch", "apply_tuning", "tune", "Mesh", "Solver", "ref_nodes", "ref_operator", "ref_sizes", "scenario_inputs",
           "solver_from_scenario"]
