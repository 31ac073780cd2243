"""GB300 (sm_103a) engine for contracting a quantum-circuit tensor network split into k partitions,
the computation that the simulated-annealing partitioner of arXiv 2507.20667 exists to speed up.

Submodules:
  tnsa     -- Python binding of the C ABI (include/tnsa.h); loads libtnsa.so, fails if missing
  inputs   -- seeded synthetic circuits and their closed tensor networks (input generation only)
  build    -- in-tree nvcc build of libtnsa.so for sm_103a
"""
__all__ = ["tnsa", "inputs", "build"]
