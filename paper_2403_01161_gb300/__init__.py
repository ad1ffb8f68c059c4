"""GB300-native immersed-boundary lattice Boltzmann droplet solver
(arXiv:2403.01161): hand-written sm_103a CUDA kernels behind the C-ABI
library ``libiblb.so`` and a thin ctypes binding (``Sim``)."""
from . import config, inputs  # noqa: F401

__all__ = ["config", "inputs"]
