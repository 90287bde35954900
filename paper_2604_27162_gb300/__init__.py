"""GB300-native batched hide-and-seek environment step (arxiv 2604.27162).

The engine is the C-ABI library ``libhase.so`` built from ``csrc/`` (CUDA for
sm_103a); ``hase`` is its thin Python binding.  Importing the package loads
nothing; the library is loaded on first use and raises if it is missing.
"""
__all__ = ["hase", "workloads"]
