"""GB300-native descent of the elastic circle-packing energy (arXiv 2303.02650).

The CUDA library (``csrc/``, C-ABI in ``include/pecc.h``) does all the work; the
``pecc`` module is a thin ctypes binding with the same names.
"""
__all__ = ["synth"]
