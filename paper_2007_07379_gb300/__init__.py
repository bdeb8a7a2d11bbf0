"""GB300-native p-bit Feynman-path sampler (arXiv 2007.07379).

Modules:
  workloads  seeded synthetic circuits and the five workloads (inputs only)
  pbits      ctypes binding of the C ABI in include/pbits.h (libpbits.so)
  build      nvcc build of libpbits.so for sm_103a
"""
__all__ = ["workloads", "pbits", "build"]
