"""Pins of the oracle's wavelet layer (Sec. 5.1: orthonormal Daubechies basis,
W^-1 maps coefficients to layer functions) against closed forms and invariants.
"""
import math
import os

import numpy as np
import pytest

from oracle import wavelets as wv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_filter_closed_forms():
    # Haar, and Daubechies' db2 / db3 closed forms (Daubechies, Ten Lectures on
    # Wavelets, Sec. 6.4): db3 uses sqrt(10) and sqrt(5 + 2 sqrt(10)).
    assert np.allclose(wv.daubechies_lowpass(1), [1 / math.sqrt(2)] * 2, atol=1e-15)
    r3 = math.sqrt(3.0)
    db2 = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * math.sqrt(2))
    assert np.abs(wv.daubechies_lowpass(2) - db2).max() < 1e-14
    s10, s = math.sqrt(10.0), math.sqrt(5 + 2 * math.sqrt(10.0))
    db3 = np.array([1 + s10 + s, 5 + s10 + 3 * s, 10 - 2 * s10 + 2 * s,
                    10 - 2 * s10 - 2 * s, 5 + s10 - 3 * s, 1 + s10 - s]) / (16 * math.sqrt(2))
    assert np.abs(wv.daubechies_lowpass(3) - db3).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_filter_conditions(p):
    h = wv.daubechies_lowpass(p)
    g = wv.highpass_from_lowpass(h)
    L = len(h)
    assert L == 2 * p
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    for m in range(p):                      # double-shift orthonormality
        dot = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert abs(dot - (1.0 if m == 0 else 0.0)) < 1e-13
    k = np.arange(L)
    for q in range(p):                      # p vanishing moments of the wavelet
        assert abs(np.sum(g * k ** q)) < 1e-9 * max(1, L ** q)
    assert abs(np.sum(h * g)) < 1e-15       # g orthogonal to h


def _read_golden(name):
    blocks, cur = [], []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            if cur:
                blocks.append(np.array(cur, dtype=float))
                cur = []
            continue
        cur.append([float(t) for t in line.split()])
    if cur:
        blocks.append(np.array(cur, dtype=float))
    return blocks


def test_haar_worked_examples():
    inp1, out1, out2 = _read_golden("haar_pyramid.txt")
    h = wv.daubechies_lowpass(1)
    assert np.allclose(wv.dwt2(inp1, h, 1), out1, atol=1e-13)
    x = np.arange(16.0).reshape(4, 4)
    assert np.allclose(wv.dwt2(x, h, 2), out2, atol=1e-13)
    assert np.allclose(wv.idwt2(out2, h, 2), x, atol=1e-13)


@pytest.mark.parametrize("p,N,J", [(3, 32, 3), (3, 16, 2), (4, 32, 2), (2, 8, 2), (3, 128, 4)])
def test_perfect_reconstruction_parseval_adjoint(p, N, J):
    rng = np.random.default_rng(N * 10 + p)
    h = wv.daubechies_lowpass(p)
    x = rng.standard_normal((N, N))
    y = rng.standard_normal((N, N))
    c = wv.dwt2(x, h, J)
    assert np.abs(wv.idwt2(c, h, J) - x).max() < 1e-12
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    # <W x, y> = <x, W^-1 y>
    assert abs(np.sum(c * y) - np.sum(x * wv.idwt2(y, h, J))) < 1e-10


def test_constant_layer_lands_in_approximation():
    # each level multiplies a constant by (sum h)^2 = 2 and leaves zero details
    h = wv.daubechies_lowpass(3)
    N, J = 32, 3
    c = wv.dwt2(np.full((N, N), 1.5), h, J)
    M = N >> J
    assert np.allclose(c[:M, :M], 1.5 * 2 ** J, atol=1e-12)
    c[:M, :M] = 0
    assert np.abs(c).max() < 1e-12


def test_vanishing_moments_in_the_pyramid():
    # db3 details of a sampled quadratic vanish away from the periodic seam
    h = wv.daubechies_lowpass(3)
    x = np.arange(64.0) ** 2
    y = wv.analysis_1d(x, h)
    d = y[32:]
    assert np.abs(d[:29]).max() < 1e-9
    assert np.abs(d[29:]).max() > 1.0      # the wrap-around seam is not a polynomial


def test_level_map():
    k = wv.level_map(8, 2)
    assert k[0, 0] == 2 and k[1, 1] == 2          # approximation -> J
    assert k[0, 2] == 2 and k[3, 3] == 2          # level-2 details
    assert k[0, 4] == 1 and k[7, 0] == 1 and k[5, 6] == 1
    assert (k == 1).sum() == 48 and (k == 2).sum() == 16
