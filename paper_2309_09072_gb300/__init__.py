"""GB300-native (sm_103a) DIST hot path of the Lu-Lin parallel LCS method.

The compute lives in a C-ABI shared library built from ``csrc/`` (see
``include/lcs.h``); :mod:`paper_2309_09072_gb300.binding` is a thin ctypes
binding with the same entry-point names.  Importing this package loads
nothing; the library is loaded on first use and raises if it is missing.
"""
__all__ = ["inputs", "binding"]
