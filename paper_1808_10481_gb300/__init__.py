"""GB300-native Hermite-leapfrog solver (arXiv 1808.10481).

The compute path is the C-ABI library ``libhl.so`` (CUDA kernels for sm_103a)
declared in ``include/hl.h``; ``paper_1808_10481_gb300.hl`` is its thin
ctypes binding.  ``paper_1808_10481_gb300.inputs`` holds the seeded synthetic
initial-data generators.  Importing the package itself loads nothing.
"""
__all__ = ["hl", "inputs"]
