"""GB300 (sm_103a) solver library for the isogeometric curl-div problem.

The compute path is the C-ABI CUDA library ``libcurldiv.so`` (sources in ``csrc/``,
declarations in ``include/curldiv.h``); ``curldiv`` is its thin ctypes binding and
``inputs`` holds the seeded synthetic input generators.  Importing the package loads
nothing; the library is loaded on first use and a missing library is an error.
"""
__all__ = ["curldiv", "inputs"]
