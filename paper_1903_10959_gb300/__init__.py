"""GB300-native ChFSI hot path of arXiv:1903.10959 (DFT-FE).

``Context`` wraps the C ABI of ``libchfsi.so`` (include/chfsi.h); every step
of the path (filter, CholGS, Rayleigh-Ritz, residuals, bounds) runs in the
library's CUDA kernels.  ``workloads`` holds the seeded synthetic inputs.
Importing this package does not load the library; constructing a Context
does, and fails loudly if it has not been built.
"""
from ._lib import (FP64, MIXED_TF32, MIXED_TF32X3, Batch, ChfsiError, Context, Server,  # noqa: F401
                   fermi_level, load)

__all__ = ["Context", "Batch", "Server", "fermi_level", "ChfsiError", "load", "FP64", "MIXED_TF32", "MIXED_TF32X3"]
