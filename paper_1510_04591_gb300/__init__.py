"""GB300-native accelerated divide-and-conquer tridiagonal eigensolver.

The compute path is the C-ABI library ``libtdeig.so`` (hand-written sm_103a
CUDA kernels); ``paper_1510_04591_gb300.tdeig`` is its thin Python binding.
Importing this package does not load the library; ``inputs`` is the seeded
workload generator and loads nothing.
"""
__all__ = ["inputs", "tdeig"]
