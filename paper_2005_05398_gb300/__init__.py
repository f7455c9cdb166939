"""GB300 (sm_103a) solver for the spline-collocation Faddeev-Merkuriev equations.

The compute path is libfm (CUDA kernels behind the C ABI of include/fm.h);
``Context`` is its ctypes binding.  Build with ``paper_2005_05398_gb300.build``.
"""
from ._lib import Context, FMError, lib, LIB_PATH  # noqa: F401

__all__ = ["Context", "FMError", "lib", "LIB_PATH"]
