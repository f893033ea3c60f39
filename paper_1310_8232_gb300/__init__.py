"""GB300-native acoustic stencil sweep (3D finite-difference "3D model" step of RTM).

Modules:
  binding    -- ctypes binding of the C-ABI library libstencil.so (same names
                as include/stencil.h); every step of the sweep runs in CUDA.
  workloads  -- seeded synthetic inputs (velocity models, shot lists, arrivals).
  build      -- compiles libstencil.so for sm_103a with nvcc.
"""
__version__ = "0.1.0"
