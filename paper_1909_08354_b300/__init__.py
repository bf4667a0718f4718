"""B300-native split-step solver of the generalized Schroedinger-Newton system.

The compute path is the CUDA library libsn.so (include/sn.h); `sn` is its
ctypes binding.  Importing this package does not load the library; the first
call into `sn` does, and fails loudly if it has not been built.
"""
from . import sn  # noqa: F401
from .sn import Grid, SNError  # noqa: F401

__all__ = ["sn", "Grid", "SNError"]
