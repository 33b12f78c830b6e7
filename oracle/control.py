"""Pseudo-open-loop control and the mirrors as the wavefront sensors see them, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages:
* Sec. 4.2: in closed loop the sensors sit behind the deformable mirrors and
  measure the residual of the incoming wavefront.  With a delay of two time
  steps, the data s measured over [t-2, t-1) belong to the mirror shapes
  a_{t-2}, the reconstruction takes [t-1, t), and a_t is applied at step t.
* Algorithm 4.1 (pseudo-open-loop control with an integrator):
  step 1, s_ol = s + A_hat a_{t-2};  step 2, Delta a = R s_ol - a_{t-2};
  step 3, a_t = a_{t-1} + g Delta a.  A_hat maps mirror shapes to the
  measurement space like the measurement operator of eq. atm_tomo, R maps
  measurements to mirror shapes, g is the gain (0.4 in Sec. 5.1).

Readings (the paper does not spell A_hat or R out):
* each mirror acts on the guide-star light like a layer at its conjugate
  altitude: sensor m sees sum_k a_k((1 - h_k/H_m) r + theta_m h_k) on its
  corners (cone factor 1 for a natural star), with the piecewise-bilinear mirror
  shapes of ``fitting``; A_hat a is then measured like layers are
  (``Tomography.measure``: Fried slopes, means for tip/tilt-only sensors);
* the residual measured with shapes a applied is measure(phi) - A_hat a;
* R is the reconstruction of one frame: the tomography solve (Sec. 5.1,
  warm-started from the previous frame's coefficients) and the fitting step
  (Sec. 4.1, warm-started from the previous frame's reconstructed commands).

Pins: tests/test_oracle_control.py (mirrors placed node for node on layers are
measured exactly as those layers; the two-step-delay integrator recursion).
"""
import math

import numpy as np

from . import atmosphere as atm
from .fitting import Fitting
from .tomography import Tomography


class Control:
    """A_hat, R and one step of Algorithm 4.1 for one geometry (with ``"fitting"``)."""

    def __init__(self, geom):
        self.tom = Tomography(geom)
        self.fit = Fitting(geom)
        self.wfs = geom["wfs"]

    def sensor_mirror_field(self, a, m):
        """sum_k a_k on the corners of sensor m (zero at inactive corners)."""
        w = self.wfs[m]
        n, d = int(w["n_sub"]), float(w["d_sub"])
        r = (np.arange(n + 1) - n / 2.0) * d
        psi = np.zeros((n + 1, n + 1))
        for k, A in enumerate(self.fit.split(a)):
            dm = self.fit.dms[k]
            c = atm.cone_factor(w, dm["altitude"])
            mid = (dm["n"] - 1) / 2.0
            gx = (c * r + w["theta"][0] * dm["altitude"]) / dm["pitch"] + mid
            gy = (c * r + w["theta"][1] * dm["altitude"]) / dm["pitch"] + mid
            for iy, wy in Fitting._taps(gy, dm["n"]):
                for ix, wx in Fitting._taps(gx, dm["n"]):
                    psi += wy[:, None] * wx[None, :] * A[np.ix_(iy, ix)]
        return psi * atm.active_corners(w["valid"])

    def mirror_slopes(self, a):
        """A_hat a: the mirrors measured by every sensor, in the slope layout."""
        out = []
        for m, w in enumerate(self.wfs):
            y = atm.fried_slopes(self.sensor_mirror_field(a, m), w["valid"])
            S = y.size // 2
            out.append(np.array([y[:S].mean(), y[S:].mean()]) if w["tt_only"] else y)
        return np.concatenate(out)

    def reconstruct(self, s, x_prev, a_prev, iters, fit_iters):
        """R s: the tomography solve from x_prev, then the fitting step from a_prev.
        Returns (coefficients, commands)."""
        x = self.tom.solve(s, x_prev, iters)
        return x, self.fit.solve(self.tom.synthesis(x), a_prev, fit_iters)

    def step(self, s, a_tm2, a_tm1, x_prev, a_rec_prev, gain, iters, fit_iters):
        """One step of Algorithm 4.1 from the residual data s measured with a_{t-2}
        applied.  Returns (a_t, coefficients, reconstructed commands R s_ol)."""
        s_ol = s + self.mirror_slopes(a_tm2)
        x, a_rec = self.reconstruct(s_ol, x_prev, a_rec_prev, iters, fit_iters)
        return a_tm1 + gain * (a_rec - a_tm2), x, a_rec
