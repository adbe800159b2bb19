"""GB300-native Laguerre-transform wave solver (Fatyanov & Terekhov, arXiv:1005.0542).

The compute path is the C-ABI library ``liblagwave.so`` (hand-written sm_103a CUDA, built by
``paper_1005_0542_gb300.build``); ``paper_1005_0542_gb300.lagwave`` is its thin ctypes binding.
``paper_1005_0542_gb300.inputs`` generates seeded synthetic workloads.  Importing the package
does not load the library; ``lagwave`` does, and raises if it is missing.
"""
__all__ = ["inputs", "lagwave", "build"]
