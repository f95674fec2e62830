"""GB300-native fused step of the double-distribution thermal lattice Boltzmann
model (Xu & Li 2022): hand-written sm_103a CUDA kernels behind the C ABI of
include/tlbm.h, with a thin ctypes binding."""
from . import tlbm  # noqa: F401
from .tlbm import Sim  # noqa: F401
