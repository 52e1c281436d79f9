"""GB300-native anti-lopsided NNLS (arXiv 1502.01645).

The solver lives in the CUDA library ``libaln`` (C ABI declared in
``include/aln.h``); ``paper_1502_01645_gb300.aln`` is its thin ctypes binding.
Importing this package does not load the library; ``aln.load()`` does, and
fails loudly when the library is missing.
"""
__all__ = ["aln", "workloads"]
