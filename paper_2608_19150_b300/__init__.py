"""B300-native implicit sweep solver for the multidimensional BGK equation.

The compute path is the CUDA library ``libbgk_b300.so`` (built from ``csrc/``), reached
through the ctypes binding in :mod:`paper_2608_19150_b300.bgk`.  Importing this package
loads nothing; :func:`paper_2608_19150_b300.bgk.load` loads the library and fails loudly
when it is missing.
"""
__all__ = ["bgk", "synth"]
