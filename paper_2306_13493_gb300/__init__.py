"""GB300 (sm_103a) implementation of the smoothed-circulant-embedding MLMC hot path.

The computation lives in the CUDA library built from csrc/ (C ABI in
include/sce.h); ``sce`` is its ctypes binding and ``build`` compiles it.
"""
from . import sce  # noqa: F401
