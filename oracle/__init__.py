"""Plain FP64 CPU oracle of the thermal MRT lattice-Boltzmann model
(arXiv:1809.08683).  TEST INFRASTRUCTURE ONLY: imported by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg, never by the
CUDA package."""
from .oracle import Oracle, build, matrix_M, matrix_Minv  # noqa: F401
