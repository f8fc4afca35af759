"""GB300-native matrix-free compressible neo-Hookean elasticity (arXiv 2505.15535).

The compute path is the CUDA library libnhmf.so (C ABI in include/nhmf.h); `nhmf` is its
thin ctypes binding.  PyTorch supplies device memory and streams only.
"""
from .nhmf import *  # noqa: F401,F403
