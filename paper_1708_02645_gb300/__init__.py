"""GB300-native periodic tricubic B-spline orbital evaluation (arXiv 1708.02645).

The compute path is the C-ABI library ``libspo.so`` (hand-written CUDA for
sm_103a); ``paper_1708_02645_gb300.spo`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use and
a missing library raises an error (there is no CPU fallback).
"""
__all__ = ["spo", "inputs"]
