"""GB300-native DCF-PCA (distributed robust PCA by consensus factorisation).

The compute path lives in the CUDA/C library ``libdcf.so`` built from
``csrc/``; :mod:`.dcf` is a thin ctypes binding with the same entry-point
names as ``include/dcf.h``.  Importing this package does not load the
library; the binding loads it on first use and raises if it is missing.
"""
__all__ = ["synth"]
