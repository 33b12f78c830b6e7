"""Orthonormal Daubechies filters and the periodic 2-D Mallat pyramid, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 5.1 chooses the compactly supported orthonormal Daubechies basis
with n = 3 (three vanishing moments, six taps) and writes the forward operator
as Gamma P W^-1, with W^-1 the inverse wavelet transform (operator expansion
after eq. eqn_lse).  The coefficient vector c_l of a layer is its wavelet
decomposition (Sec. 3, eq. REG_WAV_penalty_discr).  The paper gives no
discretisation of W; this oracle reads it as the periodic separable discrete
wavelet transform of the layer grid values (Mallat pyramid, rows then columns,
recursing on the low-low block).

Pins: tests/test_oracle_wavelets.py (filter closed forms for n = 1, 2, 3,
orthonormality and moment conditions, perfect reconstruction, Parseval,
adjointness, a hand-worked Haar example, constant fields).
"""
from math import comb, sqrt

import numpy as np


def daubechies_lowpass(p):
    """Low-pass filter h (2p taps, sum sqrt(2)) of the Daubechies wavelet with p
    vanishing moments, by spectral factorisation.

    |m0|^2 = cos^(2p)(w/2) * P(sin^2(w/2)) with P(y) = sum_{k<p} C(p-1+k, k) y^k.
    Each root y_k of P gives a root pair z, 1/z of z^2 - (2 - 4 y_k) z + 1; the
    root inside the unit circle is kept.  h holds the coefficients of
    (1 + z)^p * prod_k (z - z_k) in descending powers, scaled to sum sqrt(2)
    (this ordering gives the classical tables, e.g. db2 = (1+sqrt3, 3+sqrt3,
    3-sqrt3, 1-sqrt3)/(4 sqrt2)).
    """
    if p < 1:
        raise ValueError("p >= 1")
    poly = np.array([1.0 + 0.0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    if p > 1:
        P_desc = [float(comb(p - 1 + k, k)) for k in range(p)][::-1]
        for y in np.roots(P_desc):
            b = 2.0 - 4.0 * y
            disc = np.sqrt(b * b - 4.0 + 0.0j)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            z = z1 if abs(z1) < 1.0 else z2
            poly = np.convolve(poly, [1.0, -z])
    h = np.real(poly)
    return h * (sqrt(2.0) / h.sum())


def highpass_from_lowpass(h):
    """Quadrature mirror high-pass g_k = (-1)^k h_{Lf-1-k}."""
    Lf = len(h)
    return np.array([(-1.0) ** k * h[Lf - 1 - k] for k in range(Lf)])


def analysis_1d(x, h, axis=-1):
    """One periodic analysis level along ``axis``:
    a_i = sum_k h_k x_{(2i+k) mod M},  d_i = sum_k g_k x_{(2i+k) mod M};
    output [a_0..a_{M/2-1}, d_0..d_{M/2-1}]."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    M = x.shape[-1]
    g = highpass_from_lowpass(h)
    i = np.arange(M // 2)
    a = np.zeros(x.shape[:-1] + (M // 2,))
    d = np.zeros_like(a)
    for k in range(len(h)):
        xk = x[..., (2 * i + k) % M]
        a += h[k] * xk
        d += g[k] * xk
    return np.moveaxis(np.concatenate([a, d], axis=-1), -1, axis)


def synthesis_1d(y, h, axis=-1):
    """Transpose of ``analysis_1d`` (its inverse, the filters being orthonormal):
    x_{(2i+k) mod M} += h_k a_i + g_k d_i."""
    y = np.moveaxis(np.asarray(y, dtype=np.float64), axis, -1)
    M = y.shape[-1]
    g = highpass_from_lowpass(h)
    a, d = y[..., : M // 2], y[..., M // 2:]
    i = np.arange(M // 2)
    x = np.zeros(y.shape)
    for k in range(len(h)):
        x[..., (2 * i + k) % M] += h[k] * a + g[k] * d
    return np.moveaxis(x, -1, axis)


def dwt2(phi, h, J):
    """Analysis W: layer grid (row index = y) -> pyramid of wavelet coefficients.

    Level k acts on the top-left block of side M = N / 2^(k-1): rows (x) first,
    then columns (y).  Afterwards the block's quadrants are: top-left LL (next
    level's input), top-right high-x/low-y, bottom-left low-x/high-y,
    bottom-right high/high.
    """
    c = np.array(phi, dtype=np.float64, copy=True)
    M = c.shape[0]
    for _ in range(J):
        blk = analysis_1d(c[:M, :M], h, axis=1)
        c[:M, :M] = analysis_1d(blk, h, axis=0)
        M //= 2
    return c


def idwt2(c, h, J):
    """Synthesis W^-1 = W^T: pyramid -> layer grid (undoes ``dwt2`` level by level)."""
    phi = np.array(c, dtype=np.float64, copy=True)
    N = phi.shape[0]
    M = N >> (J - 1)
    for _ in range(J):
        blk = synthesis_1d(phi[:M, :M], h, axis=0)
        phi[:M, :M] = synthesis_1d(blk, h, axis=1)
        M *= 2
    return phi


def level_map(N, J):
    """Decomposition level k of each pyramid entry: the detail bands of level k
    occupy max(row, col) in [N/2^k, N/2^(k-1)); the final approximation block
    (max < N/2^J) is assigned level J."""
    r = np.arange(N)
    m = np.maximum(r[:, None], r[None, :])
    k = np.full((N, N), J, dtype=np.int64)
    for lev in range(1, J + 1):
        k[(m >= N >> lev) & (m < N >> (lev - 1))] = lev
    return k
