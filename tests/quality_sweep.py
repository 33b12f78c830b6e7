"""The regularisation-weight sweep of the quality metric (Sec. 5.2, the role of
alpha; Sec. 5.1, residual RMS over the evaluation directions), shared by the
oracle test and the GPU test.

A small MCAO system (8 m, two cone-compressed LGS with tip/tilt removal, one
tip/tilt-only and one full NGS, three layers of 32^2, db3 J=2) with the fitting
step onto three mirrors over 3 x 3 directions.  Each frame's truth is a seeded
von Karman atmosphere; its slopes are the noise-free measurement plus the
sensors' noise.  For each alpha the layers are reconstructed with 20 PCG
iterations (far enough towards the MAP solution that the curve shows the prior
and not the early stopping of a short solve), fitted with 4 CG iterations, and
the correction is scored against the truth by the piston-removed residual RMS
averaged over the directions.
"""
import numpy as np

from oracle import Fitting, Tomography
from synth import configs, FrozenFlow, gaussian_noise

ALPHAS = (0.2, 1.0, 2.0, 10.0, 40.0)
ITERS = 20
FIT_ITERS = 4
FRAMES = 2


def geometry(alpha=1.0, precision=0):
    g = configs.with_fitting(configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2,
                                                      precision=precision),
                             altitudes=(0.0, 4000.0, 9000.0), field_arcmin=1.2, n_dir=3)
    return dict(g, alpha=float(alpha))


def frame(k):
    """Truth layers (list of N x N) and slopes of frame k."""
    g = geometry()
    truth = FrozenFlow(g, 7, instance=k).layers(0.0)
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in g["wfs"]])
    s = Tomography(g).measure(truth) + gaussian_noise(len(sig), 1.0, 555 + k) * sig
    return truth, s


def oracle_point(alpha, truth, s, iters=ITERS):
    """The oracle's reconstruction, fit and residual RMS per direction at alpha."""
    g = geometry(alpha)
    tom, fit = Tomography(g), Fitting(g)
    x = tom.pcg(tom.rhs(s), np.zeros(tom.n), iters, tom.jacobi_diagonal())
    a = fit.solve(tom.synthesis(x), iters=FIT_ITERS)
    return x, a, fit.residual_rms(truth, a)
