"""GB300-native thermal MRT lattice-Boltzmann hot path (arXiv:1809.08683).

Submodules are imported lazily: ``lbm`` (the C-ABI binding, requires the
compiled CUDA library), ``workloads`` (seeded synthetic problems)."""
__all__ = ["lbm", "workloads"]
