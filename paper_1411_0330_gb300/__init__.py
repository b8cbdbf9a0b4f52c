"""GB300-native Lippmann-Schwinger homogenisation (Brisard & Legoll, arXiv:1411.0330).

The compute path is the CUDA library ``liblsh.so`` (sm_103a) behind the C ABI
declared in ``include/lsh.h``; ``paper_1411_0330_gb300.lsh`` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library
on first use and raises if it is missing.
"""
