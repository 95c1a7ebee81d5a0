"""GB300-native brute-force k-nearest-neighbour search (sm_103a).

The compute path is a C-ABI shared library of hand-written CUDA kernels
(``csrc/``, declared in ``include/knn.h``); ``knn.py`` is a thin ctypes
binding with the same names.  Importing this package does not load the
library; ``paper_0804_1448_gb300.knn`` does.
"""
