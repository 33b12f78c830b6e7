"""Wavelet-domain MAP tomography: noise weighting, prior, normal operator,
modified Jacobi diagonal and (P)CG, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed here:
* Sec. 2.2, eq. REG_REG_map: MAP estimate with C_Phi = diag(C_1..C_L).
* Sec. 3, D_l = diag((1/c_rho(h)) (K_out^(-11/3) + 2^((11/3) j))) and
  eq. REG_WAV_penalty_discr: the prior is diagonal in the wavelet basis.
* Sec. 4.3: block-diagonal noise covariance, sigma^2 I per natural-guide-star
  sensor; eq. removing_tt / eq. widehatc: the tip/tilt of each LGS sensor is
  removed, C_hat^-1 = (I - T) C_tilde^-1 (I - T) with T the orthogonal
  projection onto tip and tilt.
* Sec. 5.1, eq. eqn_lse: (A~^T C^-1 A~ + alpha D) c = A~^T C^-1 s, with the
  left-hand side expanded as a sum over the LGS (with C_hat) and NGS
  (with C_tilde) sensors of (Gamma P W^-1)^T C^-1 (Gamma P W^-1), plus alpha D.
* Sec. 5.1: modified Jacobi preconditioner
  J = diag(sum over LGS of A~_m^T C_tilde_m^-1 A~_m) + alpha D (no tip/tilt
  removal, NGS left out), CG/PCG, warm restart from the previous solution.

Readings where the paper is silent (each is listed in the design notes):
* the level index j of D is read as the physical frequency of level k of the
  pyramid: D = prior_weight * (L0^(-11/3) + (2^k dx)^(-11/3)), the final
  approximation block taking k = J; L0 <= 0 drops the L0 term;
* a tip/tilt-only natural guide star measures the two means of the
  full-resolution Fried slopes of its sensor, with noise sigma^2 I_2;
* spot elongation (Sec. 4.3, eq. elongation_matrix): an LGS subaperture's
  noise block is sigma^2 (I + tau g g^T) with g = beta / f the elongation
  vector in units of the spot's FWHM, read as growing linearly with the
  subaperture centre's distance from the laser launch point:
  g = elong_scale * (r - llt); natural guide stars have none; the modified
  Jacobi diagonal keeps sigma^-2 I blocks (a preconditioner only);
* CG is Hestenes-Stiefel for exactly ``iters`` iterations.

Pins: tests/test_oracle_solver.py (SPD-ness, a dense Cholesky solve that CG must
reach, CG orthogonality and residual invariants, three independent routes to
the Jacobi diagonal, closed forms of D, projection properties of I - T).
"""
import math

import numpy as np

from . import atmosphere as atm
from . import wavelets as wv


class Tomography:
    """The discrete problem for one geometry (see ``synth.configs`` for the dict)."""

    def __init__(self, geom):
        self.geom = geom
        self.h = wv.daubechies_lowpass(int(geom["wavelet_order"]))
        self.J = int(geom["levels"])
        self.alpha = float(geom["alpha"])
        self.layers = geom["layers"]
        self.wfs = geom["wfs"]
        for w in self.wfs:
            if w["tt_only"] and w["remove_tt"]:
                raise ValueError("a tip/tilt-only sensor cannot also remove tip/tilt")
        self.sizes = [lay["N"] * lay["N"] for lay in self.layers]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(int)
        self.n = int(self.offsets[-1])
        self.S = [int(np.asarray(w["valid"], bool).sum()) for w in self.wfs]
        self.n_meas = [2 if w["tt_only"] else 2 * S for w, S in zip(self.wfs, self.S)]
        self.meas_offsets = np.concatenate([[0], np.cumsum(self.n_meas)]).astype(int)
        self.D = self.prior_diagonal()

    # ------------------------------------------------------------------ layout
    def split(self, c):
        """Coefficient (or layer) vector -> list of [N, N] blocks."""
        return [np.asarray(c[o:o + s], dtype=np.float64).reshape(lay["N"], lay["N"])
                for o, s, lay in zip(self.offsets, self.sizes, self.layers)]

    def join(self, blocks):
        return np.concatenate([np.asarray(b, dtype=np.float64).ravel() for b in blocks])

    # ---------------------------------------------------------------- wavelets
    def synthesis(self, c):
        """W^-1: coefficients -> layer grids."""
        return [wv.idwt2(b, self.h, self.J) for b in self.split(c)]

    def analysis(self, phis):
        """W: layer grids -> coefficient vector."""
        return self.join([wv.dwt2(p, self.h, self.J) for p in phis])

    # ------------------------------------------------------------------- prior
    def prior_diagonal(self):
        """D (without alpha): prior_weight_l * (L0^(-11/3) + (2^k dx_l)^(-11/3))."""
        L0 = float(self.geom["L0"])
        l0_term = L0 ** (-11.0 / 3.0) if L0 > 0 else 0.0
        out = []
        for lay in self.layers:
            k = wv.level_map(lay["N"], self.J)
            out.append(lay["prior_weight"] * (l0_term + (2.0 ** k * lay["dx"]) ** (-11.0 / 3.0)))
        return self.join(out)

    # ------------------------------------------------------- forward / adjoint
    def wfs_slopes(self, m, phis):
        """Full-resolution Fried slopes Gamma_m P_m phi of sensor m."""
        w = self.wfs[m]
        return atm.fried_slopes(atm.raytrace(phis, w, self.layers), w["valid"])

    def wfs_slopes_adjoint(self, m, e):
        """P_m^T Gamma_m^T e (list of layer grids)."""
        w = self.wfs[m]
        return atm.raytrace_adjoint(atm.fried_adjoint(e, w["valid"]), w, self.layers)

    def measure(self, phis):
        """Noise-free measurement A phi (eq. atm_tomo): per sensor [sx, sy] of the
        valid subapertures, or [mean sx, mean sy] for a tip/tilt-only sensor."""
        out = []
        for m, w in enumerate(self.wfs):
            y = self.wfs_slopes(m, phis)
            S = self.S[m]
            out.append(np.array([y[:S].mean(), y[S:].mean()]) if w["tt_only"] else y)
        return np.concatenate(out)

    def _remove_tt(self, y, S):
        """(I - T) y: subtract the mean x- and mean y-slope."""
        return np.concatenate([y[:S] - y[:S].mean(), y[S:] - y[S:].mean()])

    def elongation(self, m):
        """(g_x, g_y) per valid subaperture of sensor m (row-major), or None when its
        noise is sigma^2 I: LGS sensors with elong_tau > 0 only."""
        w = self.wfs[m]
        tau = float(w.get("elong_tau", 0.0))
        if tau <= 0.0 or not (math.isfinite(float(w["height"])) and float(w["height"]) > 0) or w["tt_only"]:
            return None
        n, d = int(w["n_sub"]), float(w["d_sub"])
        b, a = np.nonzero(np.asarray(w["valid"], bool))          # row-major: b = row (y), a = column (x)
        cx, cy = (a + 0.5 - n / 2.0) * d, (b + 0.5 - n / 2.0) * d
        lx, ly = w.get("llt", (0.0, 0.0))
        eps = float(w.get("elong_scale", 0.0))
        return eps * (cx - lx), eps * (cy - ly)

    def noise_inverse_apply(self, m, y):
        """C_tilde_m^-1 y: per subaperture the 2x2 block sigma^2 (I + tau g g^T)
        (eq. elongation_matrix), solved as written; sigma^-2 y without elongation."""
        w, S = self.wfs[m], self.S[m]
        y = np.asarray(y, dtype=np.float64)
        el = self.elongation(m)
        if el is None:
            return y / w["sigma"] ** 2
        tau = float(w["elong_tau"])
        gx, gy = el
        C = np.empty((S, 2, 2))
        C[:, 0, 0] = 1.0 + tau * gx * gx
        C[:, 0, 1] = C[:, 1, 0] = tau * gx * gy
        C[:, 1, 1] = 1.0 + tau * gy * gy
        C *= w["sigma"] ** 2
        z = np.linalg.solve(C, np.stack([y[:S], y[S:]], axis=1)[..., None])[..., 0]
        return np.concatenate([z[:, 0], z[:, 1]])

    def weight_model(self, m, y):
        """Sensor m's block of C^-1 acting on model slopes y = Gamma_m P_m phi,
        returned in full-resolution slope space (so Gamma_m^T applies next)."""
        w, S = self.wfs[m], self.S[m]
        inv = 1.0 / (w["sigma"] ** 2)
        if w["tt_only"]:
            t = inv * np.array([y[:S].mean(), y[S:].mean()])     # sigma^-2 M y
            return np.concatenate([np.full(S, t[0] / S), np.full(S, t[1] / S)])  # M^T
        if w["remove_tt"]:
            # (I - T) C_tilde^-1 (I - T) y
            return self._remove_tt(self.noise_inverse_apply(m, self._remove_tt(y, S)), S)
        return self.noise_inverse_apply(m, y)

    def weight_data(self, m, s_m):
        """Sensor m's block of C^-1 applied to measured data s_m."""
        w, S = self.wfs[m], self.S[m]
        inv = 1.0 / (w["sigma"] ** 2)
        if w["tt_only"]:
            return np.concatenate([np.full(S, inv * s_m[0] / S), np.full(S, inv * s_m[1] / S)])
        s_m = np.asarray(s_m, dtype=np.float64)
        if w["remove_tt"]:
            return self._remove_tt(self.noise_inverse_apply(m, self._remove_tt(s_m, S)), S)
        return self.noise_inverse_apply(m, s_m)

    def apply_normal(self, c):
        """A_op c = W sum_m P_m^T Gamma_m^T C_m^-1 Gamma_m P_m W^-1 c + alpha D c."""
        phis = self.synthesis(c)
        g = [np.zeros((lay["N"], lay["N"])) for lay in self.layers]
        for m in range(len(self.wfs)):
            e = self.weight_model(m, self.wfs_slopes(m, phis))
            for l, gl in enumerate(self.wfs_slopes_adjoint(m, e)):
                g[l] += gl
        return self.analysis(g) + self.alpha * self.D * np.asarray(c, dtype=np.float64)

    def rhs(self, s):
        """b = W sum_m P_m^T Gamma_m^T C_m^-1 s_m (eq. eqn_lse, right-hand side)."""
        s = np.asarray(s, dtype=np.float64)
        g = [np.zeros((lay["N"], lay["N"])) for lay in self.layers]
        for m in range(len(self.wfs)):
            s_m = s[self.meas_offsets[m]:self.meas_offsets[m + 1]]
            e = self.weight_data(m, s_m)
            for l, gl in enumerate(self.wfs_slopes_adjoint(m, e)):
                g[l] += gl
        return self.analysis(g)

    # -------------------------------------------------------- Jacobi diagonal
    def _basis_profiles(self, N, k):
        """1-D periodic basis functions of level k on N samples: row c is the
        function of coefficient c of the level-k block (c < N/2^k: scaling
        function at position c, else wavelet at position c - N/2^k)."""
        M = N >> (k - 1)
        P = np.zeros((M, N))
        for c in range(M):
            x = np.zeros(N)
            x[c] = 1.0
            size = M
            while size <= N:
                x[:size] = wv.synthesis_1d(x[:size], self.h)
                size *= 2
            P[c] = x
        return P

    @staticmethod
    def _interp_1d(prof, g, N):
        """Linear interpolation (periodic) of each row of ``prof`` at coordinates g."""
        i0 = np.floor(g).astype(np.int64)
        f = g - i0
        return (1 - f) * prof[:, i0 % N] + f * prof[:, (i0 + 1) % N]

    def jacobi_diagonal(self):
        """J = diag(sum_{m LGS} sigma_m^-2 (Gamma_m P_m W^-1)^T (Gamma_m P_m W^-1)) + alpha D.

        Route: each basis function of the separable pyramid is u(x) v(y) and the
        corner coordinates are separable, so P_m w = U(a) V(b) and the Fried
        slopes are sx = dU(a) mV(b), sy = mU(a) dV(b) (d = forward difference,
        m = two-point mean); the squared norm over the valid subapertures is
        then a pair of small matrix products per level.
        """
        out = []
        for lay in self.layers:
            N = lay["N"]
            kmap = wv.level_map(N, self.J)
            Jl = np.zeros((N, N))
            for k in range(1, self.J + 1):
                prof = self._basis_profiles(N, k)
                M = prof.shape[0]
                acc = np.zeros((M, M))
                for w in self.wfs:
                    if not atm.is_lgs(w):
                        continue
                    gx, gy = atm.corner_grid_coords(w, lay)
                    U = self._interp_1d(prof, gx, N)
                    V = self._interp_1d(prof, gy, N)
                    dU, mU = U[:, 1:] - U[:, :-1], 0.5 * (U[:, 1:] + U[:, :-1])
                    dV, mV = V[:, 1:] - V[:, :-1], 0.5 * (V[:, 1:] + V[:, :-1])
                    valid = np.asarray(w["valid"], dtype=np.float64)   # [b, a]
                    acc += ((mV ** 2) @ valid @ (dU ** 2).T
                            + (dV ** 2) @ valid @ (mU ** 2).T) / w["sigma"] ** 2
                sel = kmap[:M, :M] == k
                Jl[:M, :M][sel] = acc[sel]
            out.append(Jl)
        return self.join(out) + self.alpha * self.D

    def jacobi_diagonal_probe(self):
        """Same diagonal by brute force: ||sigma^-1 Gamma_m P_m W^-1 e_lambda||^2
        summed over the LGS, one unit vector at a time (tiny grids only)."""
        Jd = np.zeros(self.n)
        lgs = [m for m, w in enumerate(self.wfs) if atm.is_lgs(w)]
        for lam in range(self.n):
            e = np.zeros(self.n)
            e[lam] = 1.0
            phis = self.synthesis(e)
            Jd[lam] = sum(np.sum(self.wfs_slopes(m, phis) ** 2) / self.wfs[m]["sigma"] ** 2
                          for m in lgs)
        return Jd + self.alpha * self.D

    def dense_normal(self):
        """The normal matrix column by column (tiny grids only)."""
        A = np.zeros((self.n, self.n))
        for lam in range(self.n):
            e = np.zeros(self.n)
            e[lam] = 1.0
            A[:, lam] = self.apply_normal(e)
        return A

    # ------------------------------------------------------------------ solver
    def pcg(self, b, x0, iters, precond=None, history=None):
        """Hestenes-Stiefel (P)CG for exactly ``iters`` iterations.

        precond: None (CG) or the vector J (z = r / J).  ``history`` (a list)
        receives (x, r, z, p, alpha, beta) per iteration when given.
        """
        b = np.asarray(b, dtype=np.float64)
        x = np.array(x0, dtype=np.float64, copy=True)
        r = b - self.apply_normal(x)
        z = r / precond if precond is not None else r.copy()
        p = z.copy()
        rz = float(r @ z)
        for _ in range(iters):
            q = self.apply_normal(p)
            pq = float(p @ q)
            if pq == 0.0 and rz == 0.0:
                a = 0.0                      # r = 0: the iterate is exact, CG stops moving
            elif not pq > 0.0:
                raise FloatingPointError("p.Ap <= 0: operator not positive definite")
            else:
                a = rz / pq
            x = x + a * p
            r = r - a * q
            z = r / precond if precond is not None else r.copy()
            rz_new = float(r @ z)
            beta = rz_new / rz if rz != 0.0 else 0.0
            if history is not None:
                history.append((x.copy(), r.copy(), z.copy(), p.copy(), a, beta))
            p = z + beta * p
            rz = rz_new
        return x

    def solve(self, s, x0=None, iters=None, precond=None):
        """One frame: b from the slopes, then (P)CG from x0 (zero when None)."""
        iters = int(self.geom["iters"] if iters is None else iters)
        x0 = np.zeros(self.n) if x0 is None else x0
        if precond is None and int(self.geom["precond"]) == 1:
            precond = self.jacobi_diagonal()
        return self.pcg(self.rhs(s), x0, iters, precond)
