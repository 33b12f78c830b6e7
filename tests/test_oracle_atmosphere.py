"""Pins of the oracle's ray-tracing (Sec. 2.1: eq. ngsproj and the LGS cone
projection) and Fried slope operator (eqs. SH_eq / SH_op, Fried geometry of
Sec. 5.1) against closed forms, special cases and dot tests."""
import math

import numpy as np
import pytest

from oracle import atmosphere as atm
from synth import configs


def _wfs(n=8, d=0.5, theta=(0.0, 0.0), height=math.inf, valid=None):
    return {"theta": theta, "height": height, "n_sub": n, "d_sub": d,
            "valid": np.ones((n, n), np.uint8) if valid is None else valid,
            "sigma": 0.1, "tt_only": False, "remove_tt": False}


def _linear_layer(N, dx, ax, ay, c0=0.0):
    idx = np.arange(N) - N / 2.0
    X, Y = np.meshgrid(idx * dx, idx * dx)        # X along columns
    return c0 + ax * X + ay * Y


def test_identity_sampling():
    # theta = 0, h = 0, d = dx: corners sit on nodes and P samples the layer
    N, n, dx = 16, 8, 0.5
    lay = {"altitude": 0.0, "dx": dx, "N": N}
    phi = np.random.default_rng(0).standard_normal((N, N))
    psi = atm.raytrace([phi], _wfs(n, dx), [lay])
    o = N // 2 - n // 2
    assert np.array_equal(psi, phi[o:o + n + 1, o:o + n + 1])


@pytest.mark.parametrize("height,h", [(math.inf, 3000.0), (90e3, 45e3), (90e3, 9000.0)])
def test_linear_layer_through_the_cone(height, h):
    # phi = ax x + ay y + c0 is reproduced exactly by bilinear interpolation, so
    # P gives (1 - h/H)(ax rx + ay ry) + ax tx h + ay ty h + c0 at every corner.
    N, n, d, dx = 64, 10, 0.5, 0.5
    ax, ay, c0 = 0.37, -0.81, 0.25
    theta = (2e-4, -1e-4)
    lay = {"altitude": h, "dx": dx, "N": N}
    w = _wfs(n, d, theta, height)
    psi = atm.raytrace([_linear_layer(N, dx, ax, ay, c0)], w, [lay])
    r = (np.arange(n + 1) - n / 2.0) * d
    RX, RY = np.meshgrid(r, r)
    cf = 1.0 - h / height if math.isfinite(height) else 1.0
    expect = cf * (ax * RX + ay * RY) + ax * theta[0] * h + ay * theta[1] * h + c0
    assert np.abs(psi - expect).max() < 1e-12
    # the cone factor for h = H/2 is exactly one half
    if math.isfinite(height) and h == height / 2:
        assert abs(atm.cone_factor(w, h) - 0.5) < 1e-15


def test_layers_add_up():
    rng = np.random.default_rng(1)
    lays = [{"altitude": 0.0, "dx": 0.5, "N": 32}, {"altitude": 7000.0, "dx": 0.5, "N": 32}]
    phis = [rng.standard_normal((32, 32)) for _ in lays]
    w = _wfs(8, 0.5, (1e-4, 2e-4), 90e3)
    both = atm.raytrace(phis, w, lays)
    sep = atm.raytrace([phis[0]], w, lays[:1]) + atm.raytrace([phis[1]], w, lays[1:])
    assert np.abs(both - sep).max() < 1e-13


def test_fried_closed_forms():
    n, d = 6, 0.5
    valid = np.ones((n, n), np.uint8)
    valid[0, 0] = 0
    r = (np.arange(n + 1) - n / 2.0) * d
    RX, RY = np.meshgrid(r, r)
    # constant phase -> zero slopes
    assert np.abs(atm.fried_slopes(np.full((n + 1, n + 1), 3.0), valid)).max() == 0.0
    # linear phase (tip/tilt) -> (ax d, ay d) on every valid subaperture
    s = atm.fried_slopes(0.7 * RX - 0.2 * RY, valid)
    S = int(valid.sum())
    assert np.allclose(s[:S], 0.7 * d, atol=1e-14) and np.allclose(s[S:], -0.2 * d, atol=1e-14)
    # bilinear phase x*y -> the gradient at the subaperture centre times d
    s = atm.fried_slopes(RX * RY, valid)
    c = (np.arange(n) + 0.5 - n / 2.0) * d
    CX, CY = np.meshgrid(c, c)
    m = valid.astype(bool)
    assert np.allclose(s[:S], (CY * d)[m], atol=1e-14)
    assert np.allclose(s[S:], (CX * d)[m], atol=1e-14)


def test_slopes_order_is_row_major():
    n = 4
    valid = np.ones((n, n), np.uint8)
    psi = np.zeros((n + 1, n + 1))
    psi[0, 2] = 2.0                 # corner a=2, b=0 -> raises sx of subap (1,0), lowers (2,0)
    s = atm.fried_slopes(psi, valid)
    assert s[1] == 1.0 and s[2] == -1.0 and np.count_nonzero(s[:16]) == 2


@pytest.mark.parametrize("wrap", [False, True])
def test_dot_tests(wrap):
    # <P phi, v> = <phi, P^T v> and <Gamma psi, s> = <psi, Gamma^T s> for the
    # separately written gather and scatter; includes a footprint that wraps.
    geom = configs.small_lgs_config(n_sub=8, N=32, n_layers=3, wrap=wrap)
    rng = np.random.default_rng(5)
    lays = geom["layers"]
    for w in geom["wfs"]:
        phis = [rng.standard_normal((l["N"], l["N"])) for l in lays]
        v = rng.standard_normal((w["n_sub"] + 1,) * 2) * atm.active_corners(w["valid"])
        lhs = np.sum(atm.raytrace(phis, w, lays) * v)
        rhs = sum(np.sum(p * g) for p, g in zip(phis, atm.raytrace_adjoint(v, w, lays)))
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))
        psi = rng.standard_normal((w["n_sub"] + 1,) * 2)
        S = int(np.asarray(w["valid"]).sum())
        s = rng.standard_normal(2 * S)
        lhs = np.sum(atm.fried_slopes(psi, w["valid"]) * s)
        rhs = np.sum(psi * atm.fried_adjoint(s, w["valid"]))
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


def test_fried_adjoint_of_tip_lives_on_the_pupil_edge():
    # Gamma^T 1_x telescopes to zero on interior corners (discrete divergence)
    valid = configs.pupil_mask(16, 0.5, 8.0, 0.3)
    S = int(valid.sum())
    tx = atm.fried_adjoint(np.concatenate([np.ones(S), np.zeros(S)]), valid)
    v = valid.astype(bool)
    interior = np.zeros((17, 17), bool)
    interior[1:-1, 1:-1] = v[:-1, :-1] & v[1:, :-1] & v[:-1, 1:] & v[1:, 1:]
    assert np.abs(tx[interior]).max() == 0.0
    assert np.abs(tx).sum() > 0


def test_wrap_is_periodic():
    # shifting the layer by a full period leaves the trace unchanged, and a
    # footprint across the seam reads the opposite edge
    N = 16
    lay = {"altitude": 1000.0, "dx": 0.5, "N": N}
    phi = np.random.default_rng(3).standard_normal((N, N))
    w = _wfs(4, 0.5, (0.0, 0.0))
    w2 = _wfs(4, 0.5, (N * 0.5 / 1000.0, 0.0))     # shifted by exactly N*dx
    assert np.abs(atm.raytrace([phi], w, [lay]) - atm.raytrace([phi], w2, [lay])).max() < 1e-12
