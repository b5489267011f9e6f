"""Batched Jacobi-preconditioned BiCGSTAB for per-cell chemistry Newton systems
on GB300 (sm_103a): the Block-cells solver of arXiv 2405.17363 rebuilt around a
C-ABI CUDA library (``libcampsolve.so``, declared in ``include/camp_solver.h``).

``paper_2405_17363_gb300.camp`` is the thin ctypes binding (same names as the C
ABI, torch tensors for device memory and streams); ``paper_2405_17363_gb300.build``
compiles the library.  Importing this package does not load the library.
"""

__all__ = ["camp", "build"]
