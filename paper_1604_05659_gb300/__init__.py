"""GB300-native simulator of one-way quantum computation patterns.

The simulation runs in libowqs.so (C ABI in include/owqs.h, CUDA kernels
for sm_103a); `owqs` is its ctypes binding.  Importing the package loads
nothing; `owqs.library()` loads the library and raises if it is missing.
"""
__all__ = ["owqs"]
