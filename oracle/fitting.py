"""Fitting step and deformable-mirror model, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages:
* Sec. 4.1, eq. fit_step_ideal: the mirror commands a minimise the expected
  squared difference between the correction H_theta a and the natural-guide-star
  projection P_theta phi (eq. ngsproj) of the atmosphere, integrated over the
  aperture and the field of view;
* Sec. 4.1, eq. fit_step_min: the field is sampled at directions theta_j and
  the problem becomes the minimum-norm least-squares solution of
  || H a - P phi ||_2, H and P stacking H_j and P^NGS_j;
* Sec. 5.1 (numerical setup): three mirrors conjugated to 0, 4 and 12.7 km,
  modelled by piecewise bilinear functions; the fitting is solved with 4 CG
  iterations over the 5 x 5 evaluation directions of the 2' square field.

Readings (the paper gives no discretisation of the aperture or the mirrors):
* the aperture is sampled at the corners of the valid subapertures of an
  n x n grid of pitch d (the Fried corner grid of a full-resolution sensor),
  every point with weight 1;
* mirror k is a square grid of n_k x n_k actuators with pitch delta_k;
  actuator (i, j) (column i = x, row j = y) sits at
  ((i - (n_k - 1)/2) delta_k, (j - (n_k - 1)/2) delta_k); its shape is
  a_k(y) = sum_ij a_k[j, i] hat(y_x/delta_k - i + (n_k-1)/2) hat(y_y/delta_k - j + (n_k-1)/2),
  hat(t) = max(0, 1 - |t|), so zero beyond the outermost actuators;
* H_j a (x) = sum_k a_k(x + h_k theta_j): science light from infinity, no cone;
* P_j phi = P^NGS_theta_j phi on the same points (``atmosphere.raytrace`` of a
  natural guide star at theta_j);
* the normal equations H^T H a = H^T P phi are solved by Hestenes-Stiefel CG,
  without preconditioner, for exactly ``iters`` iterations from a0.

Quality of a correction (Sec. 5.1, the Marechal approximation of the Strehl
ratio): in direction theta_j the residual wavefront is P_j phi - H_j a on the
sampling points; r(theta_j) is its root mean square after removing its mean
(piston does not affect the image), and s(theta_j) = exp(-(2 pi r / lambda)^2).
Readings: phases are radians at the 500 nm wavelength the screens are drawn at,
so at lambda the phase error is r * 500 nm / lambda; the paper evaluates at
2200 nm (K band).

A coefficient vector holds the mirrors concatenated, each n_k x n_k row-major.

Pins: tests/test_oracle_fitting.py (brute-force hat sums, exact reproduction of
linear mirror shapes, adjointness, zero residual when a layer is a mirror
shape, CG against the least-squares minimum).
"""
import math

import numpy as np

from . import atmosphere as atm


def hat(t):
    """The piecewise-linear hat function max(0, 1 - |t|)."""
    return np.maximum(0.0, 1.0 - np.abs(t))


class Fitting:
    """The discrete fitting problem of one geometry (``geom["fitting"]``)."""

    def __init__(self, geom):
        fit = geom["fitting"]
        self.layers = geom["layers"]
        self.dms = [dict(altitude=float(m["altitude"]), pitch=float(m["pitch"]), n=int(m["n"]))
                    for m in fit["dms"]]
        self.theta = [(float(t[0]), float(t[1])) for t in fit["directions"]]
        self.n_sub = int(fit["n_sub"])
        self.d = float(fit["d_sub"])
        self.valid = np.asarray(fit["valid"], dtype=bool)
        self.act = atm.active_corners(self.valid)
        self.iters = int(fit.get("iters", 4))
        self.sizes = [m["n"] * m["n"] for m in self.dms]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.n_points = int(self.act.sum())
        self.r = (np.arange(self.n_sub + 1) - self.n_sub / 2.0) * self.d

    def split(self, a):
        return [np.asarray(a[self.offsets[k]:self.offsets[k + 1]], dtype=np.float64).reshape(m["n"], m["n"])
                for k, m in enumerate(self.dms)]

    def dm_coords(self, k, j):
        """Actuator-grid coordinates (gx over corner columns, gy over corner rows)
        of the points x + h_k theta_j on mirror k."""
        m = self.dms[k]
        c = (m["n"] - 1) / 2.0
        gx = (self.r + m["altitude"] * self.theta[j][0]) / m["pitch"] + c
        gy = (self.r + m["altitude"] * self.theta[j][1]) / m["pitch"] + c
        return gx, gy

    @staticmethod
    def _taps(g, n):
        """The two actuators around each coordinate with their hat weights;
        indices outside 0..n-1 get weight 0 (and a clipped index)."""
        i0 = np.floor(g).astype(np.int64)
        f = g - i0
        out = []
        for i, w in ((i0, 1.0 - f), (i0 + 1, f)):
            inside = (i >= 0) & (i < n)
            out.append((np.clip(i, 0, n - 1), np.where(inside, w, 0.0)))
        return out

    def mirror(self, a, j):
        """H_j a on the corner grid [n+1, n+1] (zero at inactive corners)."""
        psi = np.zeros((self.n_sub + 1, self.n_sub + 1))
        for k, A in enumerate(self.split(a)):
            gx, gy = self.dm_coords(k, j)
            n = self.dms[k]["n"]
            for iy, wy in self._taps(gy, n):
                for ix, wx in self._taps(gx, n):
                    psi += wy[:, None] * wx[None, :] * A[np.ix_(iy, ix)]
        return psi * self.act

    def mirror_adjoint(self, u, j):
        """H_j^T u: the corner field u scattered onto the actuators with the same
        weights (np.bincount adds repeated actuator indices)."""
        u = np.asarray(u, dtype=np.float64) * self.act
        out = np.zeros(self.n)
        for k in range(len(self.dms)):
            gx, gy = self.dm_coords(k, j)
            n = self.dms[k]["n"]
            g = np.zeros(n * n)
            for iy, wy in self._taps(gy, n):
                for ix, wx in self._taps(gx, n):
                    idx = (iy[:, None] * n + ix[None, :]).ravel()
                    g += np.bincount(idx, weights=(wy[:, None] * wx[None, :] * u).ravel(), minlength=n * n)
            out[self.offsets[k]:self.offsets[k + 1]] = g
        return out

    def ngs(self, j):
        """The natural guide star of direction theta_j on the aperture sampling."""
        return {"theta": self.theta[j], "height": math.inf, "n_sub": self.n_sub, "d_sub": self.d,
                "valid": self.valid}

    def project(self, phis, j):
        """P^NGS_j phi on the corner grid (eq. ngsproj)."""
        return atm.raytrace(phis, self.ngs(j), self.layers)

    def apply_normal(self, a):
        """H^T H a = sum_j H_j^T H_j a."""
        return sum(self.mirror_adjoint(self.mirror(a, j), j) for j in range(len(self.theta)))

    def rhs(self, phis):
        """H^T P phi = sum_j H_j^T P_j phi."""
        return sum(self.mirror_adjoint(self.project(phis, j), j) for j in range(len(self.theta)))

    def residual(self, phis, a, j):
        """P_j phi - H_j a on the corner grid (zero at inactive corners)."""
        return self.project(phis, j) - self.mirror(a, j)

    def objective(self, phis, a):
        """|| H a - P phi ||_2^2 summed over the directions (eq. fit_step_min)."""
        return float(sum(np.sum(self.residual(phis, a, j) ** 2) for j in range(len(self.theta))))

    def residual_rms(self, phis, a):
        """r(theta_j) for every direction: the RMS over the sampling points of
        P_j phi - H_j a after its mean is removed (rad at 500 nm)."""
        out = np.empty(len(self.theta))
        for j in range(len(self.theta)):
            e = self.residual(phis, a, j)[self.act]
            out[j] = math.sqrt(max(0.0, float(np.mean((e - e.mean()) ** 2))))
        return out

    @staticmethod
    def strehl(rms_rad500, wavelength=2200e-9):
        """Marechal approximation exp(-(2 pi r / lambda)^2) of the Strehl ratio for a
        wavefront error of rms_rad500 radians at 500 nm, observed at `wavelength`."""
        phase = np.asarray(rms_rad500, dtype=np.float64) * (500e-9 / wavelength)
        return np.exp(-phase ** 2)

    def cg(self, b, a0, iters):
        """Hestenes-Stiefel CG on H^T H a = b for exactly ``iters`` iterations."""
        a = np.array(a0, dtype=np.float64, copy=True)
        r = np.asarray(b, dtype=np.float64) - self.apply_normal(a)
        p = r.copy()
        rr = float(r @ r)
        for _ in range(iters):
            q = self.apply_normal(p)
            pq = float(p @ q)
            if pq == 0.0 and rr == 0.0:
                alpha = 0.0
            elif not pq > 0.0:
                raise FloatingPointError("p.Hp <= 0 with a nonzero residual")
            else:
                alpha = rr / pq
            a = a + alpha * p
            r = r - alpha * q
            rr_new = float(r @ r)
            beta = rr_new / rr if rr != 0.0 else 0.0
            p = r + beta * p
            rr = rr_new
        return a

    def solve(self, phis, a0=None, iters=None):
        """The fitting step: CG on the normal equations from a0 (zero when None)."""
        a0 = np.zeros(self.n) if a0 is None else a0
        return self.cg(self.rhs(phis), a0, self.iters if iters is None else int(iters))

    def active_actuators(self):
        """Actuators whose hat support reaches a sampling point in some direction
        (the nonzero diagonal of H^T H)."""
        return int(np.count_nonzero(self.apply_normal_diagonal() > 0.0))

    def apply_normal_diagonal(self):
        """diag(H^T H) = sum_j H_j^T (weights squared)."""
        out = np.zeros(self.n)
        for j in range(len(self.theta)):
            for k in range(len(self.dms)):
                gx, gy = self.dm_coords(k, j)
                n = self.dms[k]["n"]
                g = np.zeros(n * n)
                for iy, wy in self._taps(gy, n):
                    for ix, wx in self._taps(gx, n):
                        idx = (iy[:, None] * n + ix[None, :]).ravel()
                        g += np.bincount(idx, weights=((wy[:, None] * wx[None, :]) ** 2 * self.act).ravel(),
                                         minlength=n * n)
                out[self.offsets[k]:self.offsets[k + 1]] += g
        return out

    def dense_mirror_bruteforce(self):
        """H as a dense matrix [directions x active corners, actuators], from the
        hat functions evaluated pair by pair in plain loops (tiny geometries only)."""
        b_idx, a_idx = np.nonzero(self.act)
        rows = []
        for j, (tx, ty) in enumerate(self.theta):
            for b, a in zip(b_idx, a_idx):
                x, y = self.r[a], self.r[b]
                row = np.zeros(self.n)
                for k, m in enumerate(self.dms):
                    c = (m["n"] - 1) / 2.0
                    px, py = x + m["altitude"] * tx, y + m["altitude"] * ty
                    for jj in range(m["n"]):
                        wy = max(0.0, 1.0 - abs(py / m["pitch"] - (jj - c)))
                        if wy == 0.0:
                            continue
                        for ii in range(m["n"]):
                            wx = max(0.0, 1.0 - abs(px / m["pitch"] - (ii - c)))
                            if wx != 0.0:
                                row[self.offsets[k] + jj * m["n"] + ii] += wx * wy
                rows.append(row)
        return np.array(rows)
