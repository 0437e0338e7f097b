"""GB300-native stencil sweeps (the hot path of the CharmStencil abstraction).

Submodules:
  abi     -- ctypes binding of libstencil.so, same names as include/stencil.h
  grid    -- torch-allocated buffers, Grid / Batch objects, StencilFn autograd op
  inputs  -- seeded synthetic workload inputs (no stencil arithmetic)
  build   -- nvcc build of libstencil.so for sm_103a

Importing the package loads nothing; the CUDA library is loaded on first use
and its absence is an error (there is no CPU fallback).
"""

__all__ = ["abi", "grid", "inputs", "build"]
