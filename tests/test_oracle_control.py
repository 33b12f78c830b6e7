"""Pins of the pseudo-open-loop control oracle (Sec. 4.2, Algorithm 4.1): mirrors
placed node for node on layers are measured exactly as those layers (cone
effect, tip/tilt-only means and all), and the two-step-delay integrator follows
its closed-form recursion."""
import numpy as np

from oracle import Tomography
from oracle.control import Control
from synth import configs


def _geom():
    """Two layers at the mirrors' altitudes (0 and 4 km), both on the mirrors'
    0.5 m pitch: an LGS with tip/tilt removal, a second LGS, a tip/tilt-only NGS
    and a full NGS."""
    g = configs.small_lgs_config(16, 32, 2, 2)
    return configs.with_fitting(g, altitudes=(0.0, 4000.0), pitches=(0.5, 0.5), field_arcmin=1.2, n_dir=3)


def _layers_of(ctl, g, a):
    grids = []
    for k, (m, lay) in enumerate(zip(ctl.fit.dms, g["layers"])):
        N = lay["N"]
        o = N // 2 - (m["n"] - 1) // 2
        grid = np.zeros((N, N))
        grid[o:o + m["n"], o:o + m["n"]] = a[ctl.fit.offsets[k]:ctl.fit.offsets[k + 1]].reshape(m["n"], m["n"])
        grids.append(grid)
    return grids


def test_mirrors_on_layer_nodes_are_measured_as_those_layers():
    g = _geom()
    ctl = Control(g)
    assert [m["altitude"] for m in ctl.fit.dms] == [lay["altitude"] for lay in g["layers"]]
    assert all(m["pitch"] == lay["dx"] for m, lay in zip(ctl.fit.dms, g["layers"]))
    a = np.random.default_rng(21).standard_normal(ctl.fit.n)
    got = ctl.mirror_slopes(a)
    want = Tomography(g).measure(_layers_of(ctl, g, a))
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_integrator_with_two_step_delay_follows_its_recursion():
    """A static atmosphere and a frame-independent reconstructor (cold starts):
    s_ol is the open-loop measurement every frame, R s_ol = a* is constant and
    step 3 gives e_t = e_{t-1} - g e_{t-2} for e_t = a_t - a*; from a_0 = a_1 = 0
    that is e_t = c(t) a* with c(0) = c(1) = -1.  Its characteristic roots have
    modulus sqrt(g) < 1, so the loop converges to a*."""
    g = _geom()
    ctl = Control(g)
    tom = ctl.tom
    phis = [np.random.default_rng(22 + l).standard_normal((lay["N"], lay["N"])) for l, lay in enumerate(g["layers"])]
    m = tom.measure(phis)
    gain, T = 0.4, 14
    zero_x, zero_a = np.zeros(tom.n), np.zeros(ctl.fit.n)
    _, a_star = ctl.reconstruct(m, zero_x, zero_a, 6, 4)
    a = [zero_a, zero_a]
    for t in range(2, T):
        s = m - ctl.mirror_slopes(a[t - 2])          # residual data behind the mirrors
        a_t, _, a_rec = ctl.step(s, a[t - 2], a[t - 1], zero_x, zero_a, gain, 6, 4)
        assert np.allclose(a_rec, a_star, rtol=0, atol=1e-9 * np.max(np.abs(a_star)))
        a.append(a_t)
    c = [-1.0, -1.0]
    for t in range(2, T):
        c.append(c[t - 1] - gain * c[t - 2])
    for t in range(T):
        assert np.allclose(a[t] - a_star, c[t] * a_star, rtol=0, atol=1e-8 * np.max(np.abs(a_star)))
    assert abs(c[-1]) < 2.0 * gain ** ((T - 1) / 2.0)
