"""Seeded von Karman phase screens, frozen-flow advection and measurement noise.

Screens follow the von Karman model of Sec. 3 of the paper,
m(kappa) = c_rho(h) (K_out^-2 + |kappa|^2)^(-11/6), written in the usual
textbook normalisation for phase at 500 nm with the spatial frequency f in
cycles/m:  PSD(f) = 0.023 r0_l^(-5/3) (f^2 + L0^-2)^(-11/6),
r0_l = r0 * cn2_fraction^(-3/5).  The screen is periodic on its N x N grid
(spacing dx) and has zero piston.
"""
import numpy as np


def _spectrum(N, dx, r0_layer, L0):
    f = np.fft.fftfreq(N, d=dx)
    fx, fy = np.meshgrid(f, f)                       # fx along columns (x), fy along rows (y)
    psd = 0.023 * r0_layer ** (-5.0 / 3.0) * (fx ** 2 + fy ** 2 + L0 ** -2.0) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0                                  # zero piston
    df = 1.0 / (N * dx)
    return fx, fy, np.sqrt(psd) * df


def _fourier_coefficients(N, dx, r0_layer, L0, seed):
    rng = np.random.default_rng(seed)
    fx, fy, amp = _spectrum(N, dx, r0_layer, L0)
    noise = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    return fx, fy, amp * noise


def von_karman_screen(N, dx, r0_layer, L0, seed):
    """One periodic N x N screen (float64, rad at 500 nm), row index = y."""
    _, _, F = _fourier_coefficients(N, dx, r0_layer, L0, seed)
    return np.real(np.fft.ifft2(F)) * N * N


class FrozenFlow:
    """Layers advected rigidly by their wind (Taylor frozen flow).

    The periodic screen is shifted by wind*t with an exact Fourier phase ramp,
    so every frame is again a von Karman screen on the same grid.
    """

    def __init__(self, geometry, config_id=0, instance=0, wind_seed=None):
        self.coeffs = []
        r0, L0 = geometry["r0"], geometry["L0"]
        cn2 = np.asarray(geometry["cn2"], dtype=float)
        cn2 = cn2 / cn2.sum()
        rng = np.random.default_rng(wind_seed if wind_seed is not None
                                    else 10_000 + 1000 * config_id + instance)
        for l, lay in enumerate(geometry["layers"]):
            r0_l = r0 * cn2[l] ** (-3.0 / 5.0)
            seed = 1000 * config_id + 10 * instance + l
            fx, fy, F = _fourier_coefficients(lay["N"], lay["dx"], r0_l, L0, seed)
            speed = rng.uniform(5.0, 20.0)
            ang = rng.uniform(0.0, 2.0 * np.pi)
            self.coeffs.append((fx, fy, F, speed * np.cos(ang), speed * np.sin(ang)))

    def layers(self, t):
        """Screens at time t (s): list of float64 [N, N] arrays."""
        out = []
        for fx, fy, F, vx, vy in self.coeffs:
            N = F.shape[0]
            ramp = np.exp(-2j * np.pi * (fx * vx * t + fy * vy * t))
            out.append(np.real(np.fft.ifft2(F * ramp)) * N * N)
        return out


def gaussian_noise(n, sigma, seed):
    """n samples of N(0, sigma^2) (float64) from a seeded generator."""
    return np.random.default_rng(seed).standard_normal(n) * sigma
