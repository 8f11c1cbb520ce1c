"""GB300-native (sm_103a) force evaluation of the conservative adaptive-precision
EAM+ACE potential (arxiv 2512.07693).

  build      -- compiles libapip.so (CUDA kernels + C ABI, include/apip.h)
  apip       -- ctypes binding of the C ABI (same function names)
  autograd   -- torch.autograd.Function whose backward is the library's force
  workloads  -- seeded synthetic crystals and parameters
"""
