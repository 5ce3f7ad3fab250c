"""GB300-native BOSP solver for the linear response eigenvalue problem.

The solver is a C-ABI CUDA library (include/lrep.h, include/lrep_ops.h)
built in-tree by ``paper_2506_08355_gb300.build``; ``paper_2506_08355_gb300.lrep``
is its thin ctypes binding.  ``synth`` holds the seeded input generators.
Importing the package does not load the native library; the binding loads
it on first use and raises if it is missing.
"""
__all__ = ["build", "lrep", "synth"]
