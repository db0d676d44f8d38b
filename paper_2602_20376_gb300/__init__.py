"""GB300-native (sm_103a) batched candidate scoring for low-rank discrete
quadratic maximisation (arXiv 2602.20376).

The compute path is the CUDA library ``liblrq.so`` built from ``csrc/``; the
Python module ``lrq`` is a thin ctypes binding to its C ABI (declared in
``include/lrq.h``).  ``inputs`` draws seeded synthetic workloads.
"""
__all__ = ["inputs", "lrq"]
