"""Layered-atmosphere ray-tracing and the Shack-Hartmann (Fried) slope operator, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages:
* Sec. 2.1, eq. ngsproj: a natural guide star sees sum_l phi_l(r + theta h_l).
* Sec. 2.1 (LGS projection, Fig. PF_FW_CONE): a laser guide star at altitude H
  sees sum_l phi_l((1 - h_l/H) r + theta h_l) (cone effect).
* Sec. 2.1, eqs. SH_eq / SH_op: a Shack-Hartmann sensor measures the average
  gradient over each subaperture; Sec. 5.1 discretises it in the Fried geometry.

Readings (the paper gives only the continuous maps):
* layer node (ix, iy) of an N x N grid with spacing dx sits at
  ((ix - N/2) dx, (iy - N/2) dx); values between nodes are bilinear in the node
  values, and the grid is periodic;
* corner (a, b), a, b in 0..n, of an n x n sensor with subaperture size d sits at
  ((a - n/2) d, (b - n/2) d) in the pupil;
* Fried slopes of subaperture (a, b) from its corners psi[b, a] (row = y):
  sx = (psi10 + psi11 - psi00 - psi01)/2, sy = (psi01 + psi11 - psi00 - psi10)/2
  with psi_ij = psi[b + j, a + i]: phase difference across one subaperture (rad).

Arrays: layer grids ``[N, N]`` and corner grids ``[n+1, n+1]`` are indexed
[row = y, column = x].  Slope vectors are [sx of the valid subapertures in
row-major order, then sy].

Pins: tests/test_oracle_atmosphere.py.
"""
import math

import numpy as np


def is_lgs(wfs):
    """A guide star at finite positive altitude is a laser guide star."""
    h = wfs["height"]
    return math.isfinite(h) and h > 0.0


def cone_factor(wfs, altitude):
    """1 - h/H for a laser guide star, 1 for a natural one."""
    return 1.0 - altitude / wfs["height"] if is_lgs(wfs) else 1.0


def corner_grid_coords(wfs, layer):
    """Grid coordinates (gx[a], gy[b]) on ``layer`` of the sensor corners.

    gx = ((1 - h/H) (a - n/2) d + theta_x h) / dx + N/2, likewise for y.
    """
    n, d = wfs["n_sub"], wfs["d_sub"]
    h, dx, N = layer["altitude"], layer["dx"], layer["N"]
    c = cone_factor(wfs, h)
    r = (np.arange(n + 1) - n / 2.0) * d
    gx = (c * r + wfs["theta"][0] * h) / dx + N / 2.0
    gy = (c * r + wfs["theta"][1] * h) / dx + N / 2.0
    return gx, gy


def active_corners(valid):
    """Corners belonging to at least one valid subaperture, ``[n+1, n+1]`` bool."""
    v = np.asarray(valid, dtype=bool)
    n = v.shape[0]
    act = np.zeros((n + 1, n + 1), dtype=bool)
    act[:-1, :-1] |= v
    act[1:, :-1] |= v
    act[:-1, 1:] |= v
    act[1:, 1:] |= v
    return act


def _taps(g, N):
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    return i0 % N, (i0 + 1) % N, f


def raytrace(layers_phi, wfs, layers):
    """P_m: psi[b, a] = sum_l bilinear(phi_l)(gx_l[a], gy_l[b]) on active corners."""
    n = wfs["n_sub"]
    psi = np.zeros((n + 1, n + 1))
    for phi, lay in zip(layers_phi, layers):
        gx, gy = corner_grid_coords(wfs, lay)
        x0, x1, fx = _taps(gx, lay["N"])
        y0, y1, fy = _taps(gy, lay["N"])
        phi = np.asarray(phi, dtype=np.float64)
        psi += ((1 - fy)[:, None] * ((1 - fx)[None, :] * phi[np.ix_(y0, x0)]
                                     + fx[None, :] * phi[np.ix_(y0, x1)])
                + fy[:, None] * ((1 - fx)[None, :] * phi[np.ix_(y1, x0)]
                                 + fx[None, :] * phi[np.ix_(y1, x1)]))
    return psi * active_corners(wfs["valid"])


def raytrace_adjoint(v, wfs, layers):
    """P_m^T: scatter the corner field back onto every layer grid with the same
    bilinear weights (np.bincount adds repeated node indices)."""
    v = np.asarray(v, dtype=np.float64) * active_corners(wfs["valid"])
    out = []
    for lay in layers:
        N = lay["N"]
        gx, gy = corner_grid_coords(wfs, lay)
        x0, x1, fx = _taps(gx, N)
        y0, y1, fy = _taps(gy, N)
        g = np.zeros(N * N)
        for yi, wy in ((y0, 1 - fy), (y1, fy)):
            for xi, wx in ((x0, 1 - fx), (x1, fx)):
                idx = (yi[:, None] * N + xi[None, :]).ravel()
                w = (wy[:, None] * wx[None, :] * v).ravel()
                g += np.bincount(idx, weights=w, minlength=N * N)
        out.append(g.reshape(N, N))
    return out


def fried_slopes(psi, valid):
    """Gamma_m in the Fried geometry: [sx(valid), sy(valid)], valid row-major."""
    p00, p10 = psi[:-1, :-1], psi[:-1, 1:]
    p01, p11 = psi[1:, :-1], psi[1:, 1:]
    sx = 0.5 * (p10 + p11 - p00 - p01)
    sy = 0.5 * (p01 + p11 - p00 - p10)
    m = np.asarray(valid, dtype=bool)
    return np.concatenate([sx[m], sy[m]])


def fried_adjoint(s, valid):
    """Gamma_m^T: corner field from a slope vector (scatter of the +-1/2 stencils)."""
    m = np.asarray(valid, dtype=bool)
    n = m.shape[0]
    S = int(m.sum())
    sx = np.zeros((n, n))
    sy = np.zeros((n, n))
    sx[m] = s[:S]
    sy[m] = s[S:]
    v = np.zeros((n + 1, n + 1))
    v[:-1, 1:] += 0.5 * (sx - sy)    # psi10
    v[1:, 1:] += 0.5 * (sx + sy)     # psi11
    v[:-1, :-1] += 0.5 * (-sx - sy)  # psi00
    v[1:, :-1] += 0.5 * (-sx + sy)   # psi01
    return v
