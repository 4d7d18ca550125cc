"""GB300 (sm_103a) implementation of the block epsilon-circulant all-at-once
preconditioner (Lin & Ng, arXiv 2002.01108) for backward-Euler heat equations.

The compute path is libbec.so (hand-written CUDA kernels behind the C ABI of
include/bec.h); ``bec.Problem`` is its ctypes binding.
"""
from .bec import Problem, Batch, BecError, convert, reciprocal_fp64, load, LIB_PATH, EXPORTED  # noqa: F401
