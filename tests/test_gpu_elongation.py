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

def _no_tt_removal(g):
    """The elongated blocks alone: LGS weighted by C~^-1 without (I - T)."""
    for w in g["wfs"]:
        w["remove_tt"] = False
    g["name"] += "-no-tt-removal"
    return g


CASES = {
    "small": (configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2), spot_fwhm_arcsec=0.5), 0),
    "small-fp64": (configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2, precision=1),
                                           spot_fwhm_arcsec=0.5), 0),
    "small-no-tt-removal": (_no_tt_removal(configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2),
                                                                   spot_fwhm_arcsec=0.5)), 0),
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


def test_elongation_leaves_the_jacobi_diagonal_and_tau_zero_is_bitwise_plain(lib):
    """The modified Jacobi preconditioner keeps sigma^-2 blocks (Sec. 5.1), so an elongated
    plan has the plain plan's diagonal bitwise; tau = 0 is the plain operator bitwise."""
    torch, pkg = lib
    plain = configs.small_lgs_config(16, 32, 3, 2)
    el = configs.with_elongation(plain, spot_fwhm_arcsec=0.5)
    zero = configs.with_elongation(plain, tau=0.0)
    plans = [pkg.Plan(g) for g in (plain, el, zero)]
    n = plans[0].n
    diags = []
    for p in plans:
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        p.jacobi_diagonal(d)
        diags.append(d)
    assert torch.equal(diags[0], diags[1]) and torch.equal(diags[0], diags[2])
    x = torch.tensor(np.random.default_rng(5).standard_normal(n), dtype=torch.float32, device="cuda")
    outs = []
    for p in plans:
        o = torch.empty(n, dtype=torch.float32, device="cuda")
        p.apply_normal(x, o)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[2])
    assert not torch.equal(outs[0], outs[1])
    for p in plans:
        p.close()


@pytest.mark.parametrize("C", [16, 2])
def test_batch_mixing_elongated_and_plain_is_bitwise_the_single_solves(lib, C):
    """Elongated LGS tiles carry four partials and plain ones two; a batch of both kinds
    gives each instance exactly its single solve."""
    torch, pkg = lib
    plain = configs.config1()
    geoms = [configs.with_elongation(plain), plain, configs.with_elongation(plain, tau=0.5)]
    plans = [pkg.Plan(g, cluster_size=C) for g in geoms]
    ns = plans[0].n_slopes
    s = [torch.tensor(gaussian_noise(ns, 0.3, 70 + i), dtype=torch.float32, device="cuda")
         for i in range(len(plans))]
    single = []
    for p, si in zip(plans, s):
        x = torch.zeros(p.n, dtype=torch.float32, device="cuda")
        p.solve(si, x, 5, warm=False)
        single.append(x)
    xb = [torch.zeros(p.n, dtype=torch.float32, device="cuda") for p in plans]
    pkg.solve_batch(plans, s, xb, 5, warm=False)
    torch.cuda.synchronize()
    for a, b in zip(single, xb):
        assert torch.equal(a, b)
    for p in plans:
        p.close()
