"""Pins of the oracle's noise weighting (Sec. 4.3, eqs. removing_tt / widehatc),
prior (Sec. 3), normal operator and right-hand side (Sec. 5.1, eq. eqn_lse),
modified Jacobi diagonal (Sec. 5.1) and (P)CG."""
import math

import numpy as np
import pytest

from oracle import Tomography
from oracle import atmosphere as atm
from oracle import wavelets as wv
from synth import configs


def tiny(**kw):
    args = dict(n_sub=6, N=16, n_layers=2, levels=2)
    args.update(kw)
    return configs.small_lgs_config(**args)


@pytest.fixture(scope="module")
def tiny_problem():
    t = Tomography(tiny())
    return t, t.dense_normal()


def test_prior_closed_form():
    g = tiny()
    t = Tomography(g)
    lay = g["layers"][1]
    N, dx, w = lay["N"], lay["dx"], lay["prior_weight"]
    D1 = t.D[t.offsets[1]:t.offsets[2]].reshape(N, N)
    l0 = 25.0 ** (-11.0 / 3.0)
    assert math.isclose(D1[0, 15], w * (l0 + (2 * dx) ** (-11 / 3)), rel_tol=1e-14)   # level 1
    assert math.isclose(D1[5, 2], w * (l0 + (4 * dx) ** (-11 / 3)), rel_tol=1e-14)    # level 2
    assert math.isclose(D1[1, 1], w * (l0 + (4 * dx) ** (-11 / 3)), rel_tol=1e-14)    # approx -> J
    # ratio between consecutive levels is 2^(11/3) once L0 is dropped
    g["L0"] = 0.0
    t = Tomography(g)
    D1 = t.D[t.offsets[1]:t.offsets[2]].reshape(N, N)
    assert math.isclose(D1[0, 15] / D1[5, 2], 2 ** (11 / 3), rel_tol=1e-13)
    assert (t.D > 0).all()


def _weight_matrix(t, m):
    n = 2 * t.S[m]
    return np.stack([t.weight_model(m, e) for e in np.eye(n)], axis=1)


def test_tip_tilt_removal_is_an_orthogonal_projection():
    t = Tomography(tiny())
    m = 0
    w = t.wfs[m]
    assert w["remove_tt"]
    E = _weight_matrix(t, m) * w["sigma"] ** 2       # = I - T
    assert np.abs(E - E.T).max() < 1e-15
    assert np.abs(E @ E - E).max() < 1e-14
    assert abs(np.trace(E) - (2 * t.S[m] - 2)) < 1e-12
    # it annihilates the Fried slopes of any tip/tilt (linear) phase
    n = w["n_sub"]
    r = (np.arange(n + 1) - n / 2.0) * w["d_sub"]
    RX, RY = np.meshgrid(r, r)
    s = atm.fried_slopes(1.3 * RX - 0.4 * RY, w["valid"])
    assert np.abs(E @ s).max() < 1e-13


def test_tip_tilt_only_sensor_weight():
    t = Tomography(tiny())
    m = 2
    w = t.wfs[m]
    assert w["tt_only"]
    S = t.S[m]
    E = _weight_matrix(t, m)
    M = np.zeros((2, 2 * S))
    M[0, :S] = 1.0 / S
    M[1, S:] = 1.0 / S
    assert np.abs(E - M.T @ M / w["sigma"] ** 2).max() < 1e-13
    assert np.linalg.matrix_rank(E) == 2


def test_normal_matrix_is_spd(tiny_problem):
    t, A = tiny_problem
    assert np.abs(A - A.T).max() < 1e-9 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_rhs_matches_operator_on_noise_free_data():
    # b(A W^-1 c) = A_op c - alpha D c, which ties the data weighting of each
    # sensor kind (LGS with I-T, TT-only, full NGS) to its model weighting
    t = Tomography(tiny())
    c = np.random.default_rng(2).standard_normal(t.n)
    s = t.measure(t.synthesis(c))
    assert len(s) == t.meas_offsets[-1]
    lhs = t.rhs(s)
    rhs = t.apply_normal(c) - t.alpha * t.D * c
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()


def test_cg_reaches_the_cholesky_solution():
    # a larger alpha keeps the tiny system well conditioned enough for CG to
    # reach the direct solution to 1e-9 in a few hundred iterations
    g = tiny()
    g["alpha"] = 50.0
    t = Tomography(g)
    A = t.dense_normal()
    rng = np.random.default_rng(4)
    s = t.measure(t.synthesis(rng.standard_normal(t.n))) + 0.05 * rng.standard_normal(t.meas_offsets[-1])
    b = t.rhs(s)
    L = np.linalg.cholesky(0.5 * (A + A.T))
    x_ref = np.linalg.solve(L.T, np.linalg.solve(L, b))
    Jd = t.jacobi_diagonal()
    x = t.pcg(b, np.zeros(t.n), 500, precond=Jd)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    x_cg = t.pcg(b, np.zeros(t.n), 500)
    assert np.linalg.norm(x_cg - x_ref) / np.linalg.norm(x_ref) < 1e-8


@pytest.mark.parametrize("pre", [False, True])
def test_cg_invariants(tiny_problem, pre):
    t, A = tiny_problem
    rng = np.random.default_rng(6)
    b = rng.standard_normal(t.n)
    x0 = rng.standard_normal(t.n)
    Jd = t.jacobi_diagonal() if pre else None
    hist = []
    t.pcg(b, x0, 8, precond=Jd, history=hist)
    rs = [h[1] for h in hist]
    zs = [h[2] for h in hist]
    ps = [h[3] for h in hist]
    for x, r, *_ in hist:                           # recurrence residual = true residual
        assert np.linalg.norm(r - (b - A @ x)) < 1e-9 * np.linalg.norm(b)
    for i in range(len(rs)):
        for j in range(i):
            assert abs(rs[i] @ zs[j]) < 1e-8 * np.linalg.norm(rs[i]) * np.linalg.norm(zs[j])
            assert abs(ps[i] @ A @ ps[j]) < 1e-8 * math.sqrt((ps[i] @ A @ ps[i]) * (ps[j] @ A @ ps[j]))


def test_jacobi_three_routes():
    # separable route == brute-force probing (all sensor kinds present)
    t = Tomography(tiny())
    assert np.abs(t.jacobi_diagonal() - t.jacobi_diagonal_probe()).max() < 1e-11 * t.jacobi_diagonal().max()
    # with LGS only and no tip/tilt removal, J is exactly the diagonal of the normal matrix
    g = tiny()
    g["wfs"] = [dict(w, remove_tt=False) for w in g["wfs"] if atm.is_lgs(w)]
    t = Tomography(g)
    A = t.dense_normal()
    assert np.abs(t.jacobi_diagonal() - np.diag(A)).max() < 1e-11 * np.diag(A).max()


def test_jacobi_separable_route_on_full_size_samples():
    # sampled entries at the E-ELT size (84x84, 9 layers of 128^2, J = 4) by probing
    g = configs.config1()
    t = Tomography(g)
    Jd = t.jacobi_diagonal()
    rng = np.random.default_rng(7)
    lgs = [m for m, w in enumerate(t.wfs) if atm.is_lgs(w)]
    picks = [(0, 0, 127), (8, 3, 3), (4, 70, 5), (2, 20, 40), (6, 9, 12)]
    picks += [(int(rng.integers(9)), int(rng.integers(128)), int(rng.integers(128))) for _ in range(4)]
    for l, r, c in picks:
        e = [np.zeros((128, 128)) for _ in range(9)]
        e[l][r, c] = 1.0
        phis = [wv.idwt2(x, t.h, t.J) for x in e]
        val = sum(np.sum(t.wfs_slopes(m, phis) ** 2) / t.wfs[m]["sigma"] ** 2 for m in lgs)
        lam = t.offsets[l] + r * 128 + c
        val += t.alpha * t.D[lam]
        assert math.isclose(Jd[lam], val, rel_tol=1e-11), (l, r, c)
