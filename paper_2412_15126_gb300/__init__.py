"""Encrypted ranking, order statistics and sorting under RNS-CKKS on GB300.

The compute path is the CUDA library ``librankfhe.so`` behind the C-ABI declared
in ``include/rankfhe.h``; ``paper_2412_15126_gb300.rankfhe`` is its thin ctypes
binding.  Importing this package loads nothing; importing the binding loads the
library and raises if it has not been built.
"""
