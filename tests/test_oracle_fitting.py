"""Pins of the fitting-step oracle (Sec. 4.1, eqs. fit_step_ideal / fit_step_min):
brute-force hat sums, exact reproduction of linear mirror shapes, adjointness,
a zero residual when the atmosphere is made of mirror shapes, and CG against
the dense least-squares minimum."""
import math

import numpy as np
import pytest

from oracle import Fitting
from synth import configs

ARCMIN = math.pi / (180.0 * 60.0)


def tiny(n_sub=4, N=16, dm_pitches=(0.5, 0.5), dm_alts=(0.0, 3000.0), annulus=False):
    """A tiny geometry: two layers of N^2 at 0.5 m, two mirrors, three directions."""
    d = 0.5
    D = n_sub * d
    valid = configs.pupil_mask(n_sub, d, D, 0.3) if annulus else np.ones((n_sub, n_sub), np.uint8)
    theta = [(0.0, 0.0), (0.9 * ARCMIN, -0.4 * ARCMIN), (-0.7 * ARCMIN, 0.6 * ARCMIN)]
    dms = []
    for h, p in zip(dm_alts, dm_pitches):
        R = D / 2.0 + h * 0.9 * ARCMIN
        dms.append({"altitude": h, "pitch": p, "n": 2 * int(math.ceil(R / p)) + 3})
    return {"layers": [{"altitude": h, "dx": 0.5, "N": N, "prior_weight": 1.0} for h in dm_alts],
            "fitting": {"dms": dms, "directions": theta, "n_sub": n_sub, "d_sub": d, "valid": valid,
                        "iters": 4}}


def stacked(f, grids):
    return np.concatenate([g[f.act] for g in grids])


@pytest.mark.parametrize("pitches", [(0.5, 0.5), (0.5, 0.75), (0.72, 1.0)])
def test_mirror_is_the_bruteforce_hat_sum(pitches):
    f = Fitting(tiny(dm_pitches=pitches, annulus=True))
    H = f.dense_mirror_bruteforce()
    a = np.random.default_rng(1).standard_normal(f.n)
    got = stacked(f, [f.mirror(a, j) for j in range(len(f.theta))])
    assert np.allclose(got, H @ a, rtol=0, atol=1e-13)


def test_normal_operator_and_diagonal_are_the_bruteforce_products():
    f = Fitting(tiny(dm_pitches=(0.5, 0.75)))
    H = f.dense_mirror_bruteforce()
    HtH = H.T @ H
    cols = np.array([f.apply_normal(e) for e in np.eye(f.n)]).T
    assert np.allclose(cols, HtH, rtol=0, atol=1e-12)
    assert np.allclose(f.apply_normal_diagonal(), np.diag(HtH), rtol=0, atol=1e-12)
    assert f.active_actuators() == int(np.count_nonzero(np.abs(H).sum(axis=0)))


def test_linear_mirror_shapes_are_reproduced_exactly():
    """A mirror whose actuators follow c0 + c1 x + c2 y is that plane wherever the
    points sit inside its grid: H_j a (x) = c0 + c1 (x + h theta_x) + c2 (y + h theta_y)."""
    g = tiny(dm_pitches=(0.5, 0.75), dm_alts=(0.0, 3000.0))
    f = Fitting(g)
    c0, c1, c2 = 0.3, -1.7, 0.6
    for k, m in enumerate(f.dms):
        a = np.zeros(f.n)
        c = (m["n"] - 1) / 2.0
        X = (np.arange(m["n"]) - c) * m["pitch"]
        a[f.offsets[k]:f.offsets[k + 1]] = (c0 + c1 * X[None, :] + c2 * X[:, None]).ravel()
        for j, (tx, ty) in enumerate(f.theta):
            want = c0 + c1 * (f.r[None, :] + m["altitude"] * tx) + c2 * (f.r[:, None] + m["altitude"] * ty)
            assert np.allclose(f.mirror(a, j)[f.act], want[f.act], rtol=0, atol=1e-12)


def test_mirror_adjoint_is_the_transpose():
    f = Fitting(tiny(dm_pitches=(0.72, 1.0), annulus=True))
    rng = np.random.default_rng(2)
    for j in range(len(f.theta)):
        a = rng.standard_normal(f.n)
        u = rng.standard_normal((f.n_sub + 1, f.n_sub + 1)) * f.act
        assert math.isclose(float(np.sum(f.mirror(a, j) * u)), float(a @ f.mirror_adjoint(u, j)),
                            rel_tol=1e-12)


def test_atmosphere_made_of_mirror_shapes_is_fitted_exactly():
    """Layers at the mirrors' altitudes, on the mirrors' pitch, holding the mirror
    shapes node for node: P_j phi = H_j a* in every direction (the shifts h theta_j
    and the grid conventions of P and H agree), so the objective is zero at a*
    and CG drives it to zero."""
    g = tiny(n_sub=6, N=32, dm_pitches=(0.5, 0.5), dm_alts=(0.0, 3000.0))
    f = Fitting(g)
    rng = np.random.default_rng(3)
    a_star = rng.standard_normal(f.n)
    phis = []
    for k, (m, lay) in enumerate(zip(f.dms, g["layers"])):
        N = lay["N"]
        o = N // 2 - (m["n"] - 1) // 2          # layer node of actuator 0
        grid = np.zeros((N, N))
        grid[o:o + m["n"], o:o + m["n"]] = a_star[f.offsets[k]:f.offsets[k + 1]].reshape(m["n"], m["n"])
        phis.append(grid)
    scale = sum(float(np.sum(f.project(phis, j) ** 2)) for j in range(len(f.theta)))
    assert scale > 1.0
    assert f.objective(phis, a_star) < 1e-24 * scale
    a = f.cg(f.rhs(phis), np.zeros(f.n), 200)
    assert f.objective(phis, a) < 1e-8 * scale


def test_cg_reaches_the_minimum_norm_least_squares_solution():
    g = tiny(dm_pitches=(0.5, 0.75))
    f = Fitting(g)
    H = f.dense_mirror_bruteforce()
    rng = np.random.default_rng(4)
    phis = [rng.standard_normal((16, 16)) for _ in g["layers"]]
    y = stacked(f, [f.project(phis, j) for j in range(len(f.theta))])
    a_ls = np.linalg.lstsq(H, y, rcond=None)[0]
    rank = np.linalg.matrix_rank(H)
    a = f.cg(f.rhs(phis), np.zeros(f.n), 4 * rank)
    assert np.linalg.norm(a - a_ls) < 1e-7 * np.linalg.norm(a_ls)
    assert math.isclose(f.objective(phis, a), float(np.sum((H @ a_ls - y) ** 2)), rel_tol=1e-9)


def test_cg_iterates_decrease_the_objective():
    g = tiny(dm_pitches=(0.5, 0.75), annulus=True)
    f = Fitting(g)
    rng = np.random.default_rng(5)
    phis = [rng.standard_normal((16, 16)) for _ in g["layers"]]
    b = f.rhs(phis)
    obj = [f.objective(phis, f.cg(b, np.zeros(f.n), k)) for k in range(6)]
    assert all(x1 < x0 for x0, x1 in zip(obj, obj[1:]))


def test_eelt_fitting_geometry_has_the_papers_degrees_of_freedom():
    f = Fitting(configs.with_fitting(configs.config1()))
    assert [m["altitude"] for m in f.dms] == [0.0, 4000.0, 12700.0]
    assert len(f.theta) == 25 and f.iters == 4
    assert f.active_actuators() == 9296


def test_residual_rms_ignores_piston_and_vanishes_for_a_fitted_atmosphere():
    g = tiny(n_sub=6, N=32, dm_pitches=(0.5, 0.5), dm_alts=(0.0, 3000.0))
    f = Fitting(g)
    rng = np.random.default_rng(6)
    phis = [rng.standard_normal((32, 32)) for _ in g["layers"]]
    a = rng.standard_normal(f.n)
    r = f.residual_rms(phis, a)
    assert r.shape == (3,) and np.all(r > 0)
    shifted = [phis[0] + 2.5, phis[1] - 0.7]           # piston on every layer
    assert np.allclose(f.residual_rms(shifted, a), r, rtol=1e-12, atol=0)
    for j in range(3):                                 # the RMS is numpy's standard deviation
        e = f.residual(phis, a, j)[f.act]
        assert math.isclose(r[j], float(np.std(e)), rel_tol=1e-12)
    # layers holding mirror shapes node for node: zero residual in every direction
    a_star = rng.standard_normal(f.n)
    grids = []
    for k, (m, lay) in enumerate(zip(f.dms, g["layers"])):
        o = lay["N"] // 2 - (m["n"] - 1) // 2
        grid = np.zeros((lay["N"], lay["N"]))
        grid[o:o + m["n"], o:o + m["n"]] = a_star[f.offsets[k]:f.offsets[k + 1]].reshape(m["n"], m["n"])
        grids.append(grid)
    assert np.all(f.residual_rms(grids, a_star) < 1e-12)


def test_marechal_strehl_closed_forms():
    assert Fitting.strehl(0.0) == 1.0
    # 2200/500 rad at 500 nm is 1 rad at 2200 nm: exp(-1)
    assert math.isclose(float(Fitting.strehl(2200.0 / 500.0)), math.exp(-1.0), rel_tol=1e-15)
    assert math.isclose(float(Fitting.strehl(1.0, wavelength=500e-9)), math.exp(-1.0), rel_tol=1e-15)
    s = Fitting.strehl(np.linspace(0.0, 5.0, 11))
    assert np.all(np.diff(s) < 0) and s[0] == 1.0
