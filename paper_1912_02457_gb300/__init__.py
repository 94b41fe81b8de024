"""GB300-native rotating shallow-water finite-volume scheme (arXiv 1912.02457).

The compute path is the C-ABI library ``libswe`` (hand-written sm_103a CUDA
kernels); ``paper_1912_02457_gb300.swe`` is its thin ctypes binding and
``paper_1912_02457_gb300.synth`` builds seeded synthetic workloads.
Importing this package loads nothing native; ``swe.load()`` does, and fails
loudly when the library has not been built.
"""
__all__ = ["synth", "swe"]
