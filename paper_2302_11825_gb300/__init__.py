"""GB300-native Boundary Value Caching for walk on spheres.

The compute path is the CUDA library ``libbvc.so`` (sources in ``csrc/``,
C ABI in ``include/bvc.h``); ``paper_2302_11825_gb300.bvc`` is its thin
ctypes binding.  ``paper_2302_11825_gb300.workloads`` builds seeded synthetic
inputs.  Importing this package loads nothing; the binding loads the library
on first use and raises if it is missing.
"""
__all__ = ["bvc", "workloads"]
