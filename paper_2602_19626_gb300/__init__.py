"""GB300-native per-token CDF step of a neural lossless text compressor.

The compute lives in libnc24.so (hand-written sm_103a CUDA behind the C ABI
of include/nc24.h).  ``nc24`` is the ctypes binding, ``autograd`` the torch
wrapper of the mixed-NLL backward kernel and ``build`` compiles the library.
Importing ``nc24`` fails when the library is not built; nothing here falls
back to CPU compute.
"""
__all__ = ["nc24", "autograd", "build"]
