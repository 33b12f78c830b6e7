"""Spot-elongated laser guide stars (Sec. 4.3, eq. elongation_matrix) with tip/tilt
removal (eq. widehatc) on the GPU against the FP64 oracle: the normal operator,
the right-hand side and PCG solves, through the staged gather (the analysis
kernel's shared memory) and the separate gather kernel (small clusters)."""
import numpy as np
import pytest

from oracle import Tomography
from synth import configs, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu

CASES = {
    "small": (configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2), spot_fwhm_arcsec=0.5), 0),
    "small-fp64": (configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2, precision=1),
                                           spot_fwhm_arcsec=0.5), 0),
    "eelt-C16": (configs.with_elongation(configs.config1()), 16),
    "eelt-C2": (configs.with_elongation(configs.config1()), 2),
}


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


@pytest.fixture(scope="module")
def oracles():
    return {}


def _ora(oracles, name):
    if name not in oracles:
        oracles[name] = Tomography(CASES[name][0])
    return oracles[name]


@pytest.mark.parametrize("name", list(CASES))
def test_elongated_operator_rhs_and_solve(lib, oracles, name):
    torch, pkg = lib
    g, C = CASES[name]
    ora = _ora(oracles, name)
    plan = pkg.Plan(g, cluster_size=C)
    dt = torch.float64 if g["precision"] else torch.float32
    tol = 1e-11 if g["precision"] else 1e-5
    rng = np.random.default_rng(3)
    x = rng.standard_normal(plan.n)
    out = torch.empty(plan.n, dtype=dt, device="cuda")
    plan.apply_normal(torch.tensor(x, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.apply_normal(x), f"elong-normal/{name}")
    assert e < tol, e
    s = ora.measure(ora.synthesis(rng.standard_normal(plan.n))) + gaussian_noise(plan.n_slopes, 0.3, 4)
    ds = torch.tensor(s, dtype=dt, device="cuda")
    b = torch.empty(plan.n, dtype=dt, device="cuda")
    plan.rhs(ds, b)
    b_ref = ora.rhs(s)
    e = rel(b.double().cpu().numpy(), b_ref, f"elong-rhs/{name}")
    assert e < tol, e
    xs = torch.zeros(plan.n, dtype=dt, device="cuda")
    iters = 4
    plan.solve(ds, xs, iters, warm=False)
    x_ref = ora.pcg(b_ref, np.zeros(ora.n), iters, ora.jacobi_diagonal())
    e = rel(xs.double().cpu().numpy(), x_ref, f"elong-solve/{name}")
    assert e < tol, e
    plan.close()
