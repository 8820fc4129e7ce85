"""GB300-native two-fluid (Maxwell + London + Ohmic) Yee FDTD, after arXiv 2305.13419.

  twofluid   -- ctypes binding of the C ABI in include/twofluid.h (libtwofluid.so)
  workloads  -- seeded synthetic problem descriptions (inputs only)
  build      -- in-tree nvcc build of the library for sm_103a

Submodules are imported lazily so that `workloads` can be used on machines
without the CUDA library.
"""
__all__ = ["twofluid", "workloads", "build"]
