"""GB300-native APRIL intermediate filter (arXiv 2307.01716).

The compute path lives in libapril.so (CUDA for sm_103a behind the C ABI of
include/april.h); `april` is its ctypes binding.
"""
from . import april  # noqa: F401

__all__ = ["april"]
