"""Seeded synthetic inputs shared by the CUDA path, the FP64 oracle and the benchmark.

This package holds no arithmetic of the tomography method itself (no wavelet
transform, ray-trace, slope operator, prior or solver).  It only produces the
*inputs* of the method:

* telescope/atmosphere geometries shaped like the MCAO systems of Sec. 5.1
  (guide-star asterisms, Shack-Hartmann grids and pupil masks, layer altitudes,
  grids and Cn^2 fractions, noise levels, prior weights);
* von Karman phase screens (the turbulence model of Sec. 3) drawn with a seeded
  FFT method, optionally advected by frozen flow;
* seeded white Gaussian measurement noise.

Slopes ``s = A phi + noise`` are assembled by whoever consumes these inputs
(the oracle in tests, the library's own forward operator in the benchmark),
because the forward operator is part of the method.
"""
from .configs import (config0, config1, config2, config4, small_lgs_config,
                      pupil_mask, layer_seed)
from .screens import von_karman_screen, FrozenFlow, gaussian_noise

__all__ = ["config0", "config1", "config2", "config4", "small_lgs_config",
           "pupil_mask", "layer_seed", "von_karman_screen", "FrozenFlow",
           "gaussian_noise"]
