"""GB300-native shifted Krylov (shifted COCG) solver for (z_k I - H) x^(k) = b.

The compute path is a C-ABI shared library (``libkomega_gb300.so``) built from
hand-written CUDA for sm_103a; ``paper_2001_08707_gb300.komega`` is the thin
Python binding.  Importing this package does not load the library; the binding
loads it on first use and raises if it is missing.
"""
__all__ = ["workloads", "komega", "build"]
