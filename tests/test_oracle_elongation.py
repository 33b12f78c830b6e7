"""Pins of the oracle's spot-elongated LGS noise (Sec. 4.3, eq. elongation_matrix,
with tip/tilt removal eq. widehatc): each route below is independent of the
oracle's block solve."""
import numpy as np
import pytest

from oracle import Tomography
from synth import configs


def elong_tiny(tau=0.8):
    g = configs.small_lgs_config(n_sub=6, N=16, n_layers=2, levels=2)
    return configs.with_elongation(g, tau=tau, spot_fwhm_arcsec=0.5)


def _lgs(t):
    return [m for m, w in enumerate(t.wfs) if t.elongation(m) is not None]


def test_zero_tau_is_the_plain_weighting():
    g0 = configs.small_lgs_config(n_sub=6, N=16, n_layers=2, levels=2)
    t0, t1 = Tomography(g0), Tomography(elong_tiny(tau=0.0))
    rng = np.random.default_rng(1)
    for m in range(len(t0.wfs)):
        y = rng.standard_normal(t0.n_meas[m] if t0.wfs[m]["tt_only"] else 2 * t0.S[m])
        assert np.array_equal(t0.weight_data(m, y), t1.weight_data(m, y))


def test_block_inverse_is_sherman_morrison():
    t = Tomography(elong_tiny())
    rng = np.random.default_rng(2)
    assert _lgs(t), "no elongated sensor"
    for m in _lgs(t):
        S, w = t.S[m], t.wfs[m]
        gx, gy = t.elongation(m)
        assert np.abs(gx).max() > 1.0           # elongation clearly above the spot size somewhere
        y = rng.standard_normal(2 * S)
        tau = w["elong_tau"]
        c = tau / (1.0 + tau * (gx * gx + gy * gy))
        dot = gx * y[:S] + gy * y[S:]
        ref = np.concatenate([y[:S] - c * gx * dot, y[S:] - c * gy * dot]) / w["sigma"] ** 2
        got = t.noise_inverse_apply(m, y)
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_weight_is_the_dense_projected_inverse():
    t = Tomography(elong_tiny())
    for m in _lgs(t):
        S, w = t.S[m], t.wfs[m]
        gx, gy = t.elongation(m)
        tau = w["elong_tau"]
        Cd = np.zeros((2 * S, 2 * S))
        for j in range(S):
            g = np.array([gx[j], gy[j]])
            B = w["sigma"] ** 2 * (np.eye(2) + tau * np.outer(g, g))
            Cd[np.ix_([j, S + j], [j, S + j])] = B
        one_x = np.concatenate([np.ones(S), np.zeros(S)])
        one_y = np.concatenate([np.zeros(S), np.ones(S)])
        T = (np.outer(one_x, one_x) + np.outer(one_y, one_y)) / S
        P = np.eye(2 * S) - T
        ref = P @ np.linalg.inv(Cd) @ P if w["remove_tt"] else np.linalg.inv(Cd)
        got = np.stack([t.weight_model(m, e) for e in np.eye(2 * S)], axis=1)
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
        assert np.abs(got - got.T).max() < 1e-12 * np.abs(got).max()
        assert np.linalg.eigvalsh(0.5 * (got + got.T)).min() > -1e-12 * np.abs(got).max()
        if w["remove_tt"]:
            assert np.abs(got @ one_x).max() < 1e-12 * np.abs(got).max()
            assert np.abs(got @ one_y).max() < 1e-12 * np.abs(got).max()


def test_elongated_normal_matrix_is_spd_and_cg_reaches_cholesky():
    g = elong_tiny()
    g["alpha"] = 50.0
    t = Tomography(g)
    A = t.dense_normal()
    assert np.abs(A - A.T).max() < 1e-10 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    rng = np.random.default_rng(5)
    s = t.measure(t.synthesis(rng.standard_normal(t.n))) + 0.05 * rng.standard_normal(t.meas_offsets[-1])
    b = t.rhs(s)
    Lc = np.linalg.cholesky(0.5 * (A + A.T))
    x_ref = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b))
    x = t.pcg(b, np.zeros(t.n), 600, precond=t.jacobi_diagonal())
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
