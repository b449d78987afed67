"""GB300-native 2D3V electromagnetic particle-in-cell step (arXiv 2106.12485).

The compute path is the CUDA library built from csrc/ (C ABI in
include/zpic.h); `zpic` is its ctypes binding and `workloads` builds the
configurations of the benchmark workloads.
"""
from . import zpic  # noqa: F401

__all__ = ["zpic"]
