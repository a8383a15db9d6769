"""B300-native simulator of a large mesh chip multicore joined by a bufferless,
deflection-routed NoC with an LSPD L2 (arXiv 1508.03235).

Submodules:
  inputs    -- seeded workload parameters and the batch design-point sampler
  noc       -- ctypes binding of the CUDA library libnoc.so (the product path)
  surrogate -- the BF16 tensor-core MLP surrogate trained on simulator output
The package import itself loads nothing native; import `noc` for the simulator.
"""
__all__ = ["inputs", "noc"]
