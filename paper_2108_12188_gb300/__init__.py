"""GB300-native spectral-element Poisson hot path (matrix-free Ax, gather-scatter, CG).

The compute path is libsem.so (CUDA kernels for sm_103a behind the C ABI in
include/sem.h); `sem` is its thin ctypes binding.
"""
from . import sem  # noqa: F401
from .sem import *  # noqa: F401,F403
