"""GB300-native lattice Boltzmann Maxwell solver for radiation forces and torques on
Janus cylinders (arXiv 2509.22308).  The compute path is the CUDA library built
from ``csrc/``; ``lbm_em`` is its thin ctypes binding."""
__all__ = ["lbm_em", "workloads"]
