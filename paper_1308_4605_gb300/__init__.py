"""GB300 (sm_103a) solver for the variable-coefficient staggered Stokes system
of Cai, Nonaka, Bell, Griffith & Donev (arXiv:1308.4605).

  stokes      ctypes binding of the C ABI (include/stokes.h) of
              libstokes_gb300.so; raises on import if the library is missing
  workloads   seeded synthetic coefficient fields and right-hand sides
  build       nvcc build of the shared library
"""
__all__ = ["stokes", "workloads", "build"]
