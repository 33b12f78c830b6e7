"""The quality metric as the regularisation weight varies (Sec. 5.2; Sec. 5.1's
residual RMS), on the oracle: the wavelet prior must behave sensibly.

With a reconstruction well on its way to the MAP solution, too small an alpha
lets the measurement noise and the tomographic null space through, too large an
alpha flattens the layers towards the prior mean; the residual RMS of the
correction is then smallest at a moderate alpha.  The paper finds its best
weights at alpha of 1 to 2 on its E-ELT simulations.  Measured on this
synthetic system after 20 PCG iterations (mean over two frames and the 3 x 3
directions, rad at 500 nm): alpha 0.2: 7.43, 1: 5.07, 2: 4.46, 10: 4.14,
40: 4.93; after 30 iterations the minimum moves to alpha 2 (5.36, 4.04, 3.87,
4.12, 4.86).
"""
import numpy as np

import quality_sweep as qs


def test_residual_rms_is_smallest_at_a_moderate_alpha():
    curve = {}
    for alpha in qs.ALPHAS:
        rms = []
        for k in range(qs.FRAMES):
            truth, s = qs.frame(k)
            rms.append(np.mean(qs.oracle_point(alpha, truth, s)[2]))
        curve[alpha] = float(np.mean(rms))
    assert all(np.isfinite(v) and v > 0 for v in curve.values()), curve
    best = min(curve, key=curve.get)
    assert best in (1.0, 2.0, 10.0), curve
    # the ends of the sweep are clearly worse than the best weight
    assert curve[qs.ALPHAS[0]] > 1.2 * curve[best], curve
    assert curve[qs.ALPHAS[-1]] > 1.1 * curve[best], curve
