"""Geometries of the MCAO workloads (plain data; no method arithmetic).

A geometry is a plain ``dict``:

``D_tel`` (m), ``obstruction`` (central obstruction as a *radius* ratio),
``wfs`` (list of dicts: ``theta`` = (theta_x, theta_y) in rad, ``height`` in m
(``inf`` for a natural guide star), ``n_sub``, ``d_sub`` (m), ``valid`` (uint8
array ``[n_sub, n_sub]``, row index = y subaperture index, column = x),
``sigma`` (rad per slope), ``tt_only``, ``remove_tt``),
``layers`` (list of dicts: ``altitude`` (m), ``dx`` (m), ``N``,
``prior_weight`` = 1/c_rho(h)), ``wavelet_order`` (Daubechies vanishing
moments: 3 -> 6 taps), ``levels``, ``alpha``, ``L0`` (m), ``precond``
(0 = CG, 1 = modified Jacobi PCG), ``precision`` (0 = FP32 operator with FP64
reductions, 1 = FP64), and harness keys ``iters``, ``warm``, ``cn2``, ``r0``,
``name``, ``seed_base``.

The E-ELT numbers follow Sec. 5.1 of the paper (42 m pupil, about 28 % of the
area obstructed, six sodium LGS with 84x84 Shack-Hartmann sensors, NGS used for
tip/tilt).  Ring sizes quoted as "ring" are read as diameters (a 2' ring puts
the NGS at 1' from the axis), which keeps every footprint inside the layer grid.
"""
import math

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)
SODIUM_HEIGHT = 90e3
R0_500NM = 0.15
OUTER_SCALE = 25.0

ELT_HEIGHTS = [0.0, 600.0, 1200.0, 2500.0, 5000.0, 7500.0, 10000.0, 15000.0, 20000.0]
ELT_CN2 = [0.5, 0.1, 0.1, 0.07, 0.06, 0.05, 0.05, 0.04, 0.03]


def layer_seed(config_id, instance, layer):
    """Seed of the phase screen of one layer: 1000*config + 10*instance + layer."""
    return 1000 * config_id + 10 * instance + layer


def pupil_mask(n_sub, d_sub, D_tel, obstruction=0.0):
    """Valid-subaperture mask of a circular pupil: a subaperture is valid iff its
    centre lies in the annulus ``obstruction*D/2 <= r <= D/2``.

    Returned as uint8 ``[n_sub, n_sub]`` with row = y index, column = x index.
    """
    c = (np.arange(n_sub) + 0.5 - n_sub / 2.0) * d_sub
    cx, cy = np.meshgrid(c, c)          # cx varies along columns (x), cy along rows (y)
    r = np.hypot(cx, cy)
    m = (r <= D_tel / 2.0) & (r >= obstruction * D_tel / 2.0)
    return m.astype(np.uint8)


def prior_weight(cn2_fraction, dx, r0=R0_500NM):
    """1/c_rho(h) for a layer holding ``cn2_fraction`` of the turbulence.

    c_rho is set so that the prior variance of the finest-level wavelet
    coefficients (level 1, scale 2*dx) matches the variance measured once on
    the seeded von Karman screens of this package, 0.9*(dx/r0_l)^(5/3) with
    r0_l = r0*f^(-3/5) (about a quarter of half the phase structure function at
    lag dx):  c_rho = f * 0.9*(dx/r0)^(5/3) * (2*dx)^(11/3).
    """
    c_rho = cn2_fraction * 0.9 * (dx / r0) ** (5.0 / 3.0) * (2.0 * dx) ** (11.0 / 3.0)
    return 1.0 / c_rho


def _ring(n, radius, start_deg):
    return [(radius * math.cos(math.radians(start_deg + 360.0 * k / n)),
             radius * math.sin(math.radians(start_deg + 360.0 * k / n))) for k in range(n)]


def _wfs(theta, height, n_sub, d_sub, D_tel, obstruction, sigma, tt_only=False,
         remove_tt=False):
    return {"theta": (float(theta[0]), float(theta[1])), "height": float(height),
            "n_sub": int(n_sub), "d_sub": float(d_sub),
            "valid": pupil_mask(n_sub, d_sub, D_tel, obstruction),
            "sigma": float(sigma), "tt_only": bool(tt_only), "remove_tt": bool(remove_tt)}


def _layers(heights, cn2, N, dx, r0=R0_500NM):
    tot = float(sum(cn2))
    return [{"altitude": float(h), "dx": float(dx), "N": int(N),
             "prior_weight": prior_weight(f / tot, dx, r0)} for h, f in zip(heights, cn2)]


def config0():
    """Plain method, small, FP64: 8 m, 16x16 SH, 3 NGS on a 1' ring, 2 layers of 32^2."""
    D = 8.0
    wfs = [_wfs(t, math.inf, 16, 0.5, D, 0.0, 0.1) for t in _ring(3, 0.5 * ARCMIN, 90.0)]
    return {"name": "cfg0-8m-16x16-3ngs-2x32^2-fp64", "D_tel": D, "obstruction": 0.0,
            "wfs": wfs, "layers": _layers([0.0, 6000.0], [0.7, 0.3], 32, 0.5),
            "wavelet_order": 3, "levels": 3, "alpha": 1.0, "L0": OUTER_SCALE,
            "precond": 0, "precision": 1, "iters": 30, "warm": False,
            "cn2": [0.7, 0.3], "r0": R0_500NM, "seed_base": 0}


def config1():
    """E-ELT MCAO: 42 m (28 % area obstructed), 6 LGS 84x84 at 90 km on a 1'-radius
    hexagon, 3 tip/tilt NGS at 1' radius, 9 layers of 128^2 at 0.5 m, db3 J=4,
    Jacobi PCG, 10 iterations, warm start."""
    D, obs = 42.0, math.sqrt(0.28)
    wfs = [_wfs(t, SODIUM_HEIGHT, 84, 0.5, D, obs, 0.3, remove_tt=True)
           for t in _ring(6, 1.0 * ARCMIN, 0.0)]
    wfs += [_wfs(t, math.inf, 84, 0.5, D, obs, 0.1, tt_only=True)
            for t in _ring(3, 1.0 * ARCMIN, 90.0)]
    return {"name": "cfg1-eelt-42m-84x84-6lgs-3ttngs-9x128^2", "D_tel": D,
            "obstruction": obs, "wfs": wfs,
            "layers": _layers(ELT_HEIGHTS, ELT_CN2, 128, 0.5),
            "wavelet_order": 3, "levels": 4, "alpha": 1.0, "L0": OUTER_SCALE,
            "precond": 1, "precision": 0, "iters": 10, "warm": True,
            "cn2": list(ELT_CN2), "r0": R0_500NM, "seed_base": 1000}


def _min_grid(D, wfs_list, heights, dx):
    ext = 0.0
    for w in wfs_list:
        th = max(abs(w["theta"][0]), abs(w["theta"][1]))
        for h in heights:
            c = 1.0 - h / w["height"] if math.isfinite(w["height"]) else 1.0
            ext = max(ext, th * h + c * D / 2.0)
    return 2.0 * ext / dx + 4.0


def config2(n_instances=64, seed=2000):
    """64 independent instances of uneven size (batched workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n_sub = int(rng.choice([16, 32, 40, 64, 84]))
        L = int(rng.integers(2, 10))
        m_lgs = int(rng.integers(3, 7))
        D = n_sub * 0.5
        wfs = [_wfs(t, SODIUM_HEIGHT, n_sub, 0.5, D, 0.0, 0.3, remove_tt=True)
               for t in _ring(m_lgs, 1.0 * ARCMIN, 0.0)]
        wfs += [_wfs(t, math.inf, n_sub, 0.5, D, 0.0, 0.1, tt_only=True)
                for t in _ring(3, 1.0 * ARCMIN, 90.0)]
        heights = ELT_HEIGHTS[:L]
        need = _min_grid(D, wfs, heights, 0.5)
        grids = [g for g in (32, 64, 128, 256) if g >= need]
        N = int(rng.choice(grids))
        J = min(4, int(round(math.log2(N))) - 2)
        out.append({"name": f"cfg2-inst{i}-{n_sub}x{n_sub}-{L}L-{m_lgs}lgs-{N}^2",
                    "D_tel": D, "obstruction": 0.0, "wfs": wfs,
                    "layers": _layers(heights, ELT_CN2[:L], N, 0.5),
                    "wavelet_order": 3, "levels": J, "alpha": 1.0, "L0": OUTER_SCALE,
                    "precond": 1, "precision": 0, "iters": 10, "warm": True,
                    "cn2": list(ELT_CN2[:L]), "r0": R0_500NM,
                    "seed_base": 2000 + 10 * i})
    return out


def config4(seed=4000):
    """100 m class: 200x200 SH, 9 LGS on a 1.5' ring, 3 TT NGS, 35 layers of 512^2, db4 J=5."""
    rng = np.random.default_rng(seed)
    D = 100.0
    heights = [0.0] + sorted(float(h) for h in rng.uniform(0.0, 25e3, 34))
    cn2 = [math.exp(-h / 5e3) for h in heights]
    wfs = [_wfs(t, SODIUM_HEIGHT, 200, 0.5, D, 0.0, 0.3, remove_tt=True)
           for t in _ring(9, 0.75 * ARCMIN, 0.0)]
    wfs += [_wfs(t, math.inf, 200, 0.5, D, 0.0, 0.1, tt_only=True)
            for t in _ring(3, 1.0 * ARCMIN, 90.0)]
    return {"name": "cfg4-100m-200x200-9lgs-3ttngs-35x512^2-db4", "D_tel": D,
            "obstruction": 0.0, "wfs": wfs, "layers": _layers(heights, cn2, 512, 0.5),
            "wavelet_order": 4, "levels": 5, "alpha": 1.0, "L0": OUTER_SCALE,
            "precond": 1, "precision": 0, "iters": 20, "warm": True,
            "cn2": cn2, "r0": R0_500NM, "seed_base": 4000}


def small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2, order=3, precision=0,
                     precond=1, wrap=False, full_ngs=True, d_sub=0.5, dx=0.5,
                     obstruction=0.3):
    """A small system with every feature of the operator: cone-compressed LGS
    with tip/tilt removal, a tip/tilt-only NGS and (optionally) a full-resolution
    NGS; used for parity cases that the oracle finishes in seconds.

    ``wrap=True`` shifts one guide star so that its footprint crosses the edge of
    the periodic layer grids.
    """
    D = n_sub * d_sub
    heights = [0.0, 4000.0, 9000.0, 14000.0, 6500.0][:n_layers]
    cn2 = [0.6, 0.25, 0.15, 0.1, 0.05][:n_layers]
    a = 0.6 * ARCMIN
    wfs = [_wfs((a, 0.0), SODIUM_HEIGHT, n_sub, d_sub, D, obstruction, 0.3, remove_tt=True),
           _wfs((-0.5 * a, 0.8 * a), SODIUM_HEIGHT, n_sub, d_sub, D, obstruction, 0.25,
                remove_tt=True),
           _wfs((0.3 * a, -0.9 * a), math.inf, n_sub, d_sub, D, obstruction, 0.1,
                tt_only=True)]
    if full_ngs:
        wfs.append(_wfs((-0.7 * a, -0.4 * a), math.inf, n_sub, d_sub, D, obstruction, 0.15))
    if wrap:
        # put the footprint of the first LGS across the grid edge on the top layer
        shift = (N * dx / 2.0) / max(heights)
        wfs[0]["theta"] = (shift, 0.25 * shift)
    return {"name": f"small-{n_sub}x{n_sub}-{n_layers}x{N}^2-J{levels}-db{order}"
                    f"{'-wrap' if wrap else ''}{'-fp64' if precision else ''}",
            "D_tel": D, "obstruction": obstruction, "wfs": wfs,
            "layers": _layers(heights, cn2, N, dx),
            "wavelet_order": order, "levels": levels, "alpha": 1.0,
            "L0": OUTER_SCALE, "precond": precond, "precision": precision,
            "iters": 8, "warm": True, "cn2": cn2, "r0": R0_500NM, "seed_base": 9000}


def with_elongation(geom, tau=0.8, spot_fwhm_arcsec=1.0, sodium_depth_m=10e3, launch_radius=None):
    """A copy of geom with spot elongation (Sec. 4.3, eq. elongation_matrix) on every
    laser guide star sensor: tau as in the paper's tests (0.8); a subaperture's
    elongation is the sodium layer's depth seen from the distance to the launch
    point, depth * r / H^2 rad, in units of the spot FWHM, so
    elong_scale = depth / H^2 / FWHM per metre; the lasers are launched from the pupil
    edge (launch_radius, default D/2) at their guide star's azimuth."""
    import copy
    g = copy.deepcopy(geom)
    R = g["D_tel"] / 2.0 if launch_radius is None else float(launch_radius)
    fwhm = spot_fwhm_arcsec * math.pi / 180.0 / 3600.0
    for w in g["wfs"]:
        H = float(w["height"])
        if w["tt_only"] or not (math.isfinite(H) and H > 0):
            continue
        az = math.atan2(float(w["theta"][1]), float(w["theta"][0]))
        w["elong_tau"] = float(tau)
        w["elong_scale"] = sodium_depth_m / H ** 2 / fwhm
        w["llt"] = (R * math.cos(az), R * math.sin(az))
    g["name"] = g["name"] + "-elong"
    return g



def with_fitting(geom, altitudes=(0.0, 4000.0, 12700.0), pitches=(0.5, 0.72, 1.0), field_arcmin=2.0,
                 n_dir=5, iters=4):
    """A copy of geom with the fitting step's geometry (Sec. 4.1, eq. fit_step_min;
    Sec. 5.1 setup): mirrors at ``altitudes`` with actuator ``pitches``, each a
    square grid covering the aperture seen from every direction; ``n_dir`` x
    ``n_dir`` directions on a square field of side ``field_arcmin``; the aperture
    sampled at the corners of the valid subapertures of the first full-resolution
    sensor.  The paper gives the altitudes and the total, 9296 degrees of freedom,
    not the pitches: on the E-ELT geometry the default pitches (0.5, 0.72, 1.0 m)
    give 4240 + 2856 + 2200 = 9296 actuators whose support reaches a sampling
    point."""
    import copy
    g = copy.deepcopy(geom)
    full = [w for w in g["wfs"] if not w["tt_only"]][0]
    n_sub, d = int(full["n_sub"]), float(full["d_sub"])
    half = 0.5 * field_arcmin * ARCMIN
    ts = np.linspace(-half, half, n_dir) if n_dir > 1 else np.zeros(1)
    dms = []
    for h, p in zip(altitudes, pitches):
        R = n_sub * d / 2.0 + float(h) * half
        dms.append({"altitude": float(h), "pitch": float(p), "n": 2 * int(math.ceil(R / p)) + 3})
    g["fitting"] = {"dms": dms, "directions": [(float(tx), float(ty)) for ty in ts for tx in ts],
                    "n_sub": n_sub, "d_sub": d,
                    "valid": pupil_mask(n_sub, d, g["D_tel"], g["obstruction"]), "iters": int(iters)}
    g["name"] = g["name"] + "-fit"
    return g
