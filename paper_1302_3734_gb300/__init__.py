"""GB300-native wavelet-domain MAP tomography for multi-conjugate adaptive optics.

The solve of the paper's normal equations (Helin & Yudytskiy, Sec. 5.1,
eq. eqn_lse) and the fitting step that turns its layers into mirror commands
(Sec. 4.1, eq. fit_step_min) run in hand-written sm_103a CUDA kernels behind the C ABI of
``include/tomo.h``; ``binding`` is a thin ctypes layer over it and ``build``
compiles the library in-tree.
"""
from .binding import (Plan, Fit, Server, TomoError, solve_batch, launch_count, load_library, version,
                      probe_l2_read, geometry_struct, fit_geometry_struct, SIGNATURES, LIB_PATH)

__all__ = ["Plan", "Fit", "Server", "TomoError", "solve_batch", "launch_count", "load_library", "version",
           "probe_l2_read", "geometry_struct", "fit_geometry_struct", "SIGNATURES", "LIB_PATH"]
