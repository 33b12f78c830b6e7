"""GB300-native wavelet-domain MAP tomography for multi-conjugate adaptive optics.

The solve of the paper's normal equations (Helin & Yudytskiy, Sec. 5.1,
eq. eqn_lse) runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/tomo.h``; ``binding`` is a thin ctypes layer over it and ``build``
compiles the library in-tree.
"""
from .binding import (Plan, Server, TomoError, solve_batch, launch_count, load_library, version,
                      geometry_struct, SIGNATURES, LIB_PATH)

__all__ = ["Plan", "Server", "TomoError", "solve_batch", "launch_count", "load_library", "version",
           "geometry_struct", "SIGNATURES", "LIB_PATH"]
