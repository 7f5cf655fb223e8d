"""GB300-native multilevel CC2 / CCSD hot path (arXiv 2006.05226): libmlcc and its binding.

libmlcc.so (csrc/, C ABI in include/mlcc.h) holds every kernel of the method; mlcc.py is
the ctypes binding used by the tests and the benchmark.
"""
from . import mlcc  # noqa: F401
