"""GB300-native pressure-Poisson hot path: matrix-free variable-spacing PCG
with deep-learning line-search steps (HyDEA on non-uniform grids).

The compute path is the CUDA library built from ``csrc/`` for sm_103a and
exposed through the C ABI of ``include/ppe.h``; ``api`` is its thin Python
face.  ``inputs`` draws seeded synthetic workloads.
"""
__all__ = ["api", "inputs", "build"]
