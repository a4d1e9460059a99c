"""GB300-native Larger-than-Life step (the CAT method, arXiv 2406.17284).

The compute path is the CUDA library ``libcat.so`` built from ``csrc/`` for
sm_103a and reached through the C ABI declared in ``include/cat.h``;
``paper_2406_17284_gb300.cat`` is the thin ctypes binding.  Importing this
package does not load the library (``inputs`` is usable without a GPU).
"""
__all__ = ["inputs", "cat"]
