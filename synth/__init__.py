"""Seeded synthetic chemistry workloads shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This package only *generates inputs*: mechanisms, per-cell concentrations, the
mass-action Jacobian values ``A = I - gamma*J`` on the shared CSR pattern and the
right-hand sides.  It contains no part of the linear solver.
"""
from .mechanism import (Mechanism, CellBatch, make_mechanism, make_cells,
                        workload, WORKLOADS)

__all__ = ["Mechanism", "CellBatch", "make_mechanism", "make_cells", "workload",
           "WORKLOADS"]
