"""tmamg: multi-rhs, multi-shift twisted-mass Wilson-clover solver with aggregation-based
adaptive multigrid (arXiv:2201.03872), as a CUDA library for GB300 (sm_103a).

The compute path is libtmamg.so (C ABI in include/tmamg.h); ``tmamg`` is its thin
ctypes binding. Importing this package does not load the library; the first call does.
"""
from . import tmamg  # noqa: F401
