"""GB300 (sm_103a) compatible-weighted-matching AMG coarsening (arXiv 1810.04221).

Modules:
  build     -- in-tree nvcc build of lib/libcwmamg.so (C ABI: include/cwm_amg.h)
  binding   -- ctypes binding with the C entry points' names (torch tensors in, no fallback)
  problems  -- seeded synthetic s.p.d. test matrices
Importing the package loads nothing; the CUDA library loads on first use of `binding`.
"""
__all__ = ["binding", "build", "problems"]
