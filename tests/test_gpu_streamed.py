"""Streamed transforms (tomo_plan_options.transforms = 2): W and W^-1 level by
level over row tiles of every layer, without thread-block clusters, with the
PCG epilogue and the fused direction update of the cluster kernels.  Every
operator and the fixed-iteration solve against the FP64 oracle at the
tolerances of the cluster path, on grids that use only the coarse kernel
(32^2), one pass (128^2; also Haar and db2) and two passes (256^2, db4), in FP32
and FP64; a
streamed batch of uneven plans is bitwise the plans solved alone, and the
streamed and cluster paths agree to rounding.
"""
import numpy as np
import pytest

from oracle import Tomography
from synth import configs, FrozenFlow, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu

CASES = {
    "coarse-only-32": lambda: configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2),
    "one-pass-128": lambda: configs.small_lgs_config(n_sub=40, N=128, n_layers=3, levels=3, order=3),
    "two-pass-256-db4": lambda: configs.small_lgs_config(n_sub=48, N=256, n_layers=2, levels=4, order=4),
    "one-pass-128-fp64": lambda: configs.small_lgs_config(n_sub=40, N=128, n_layers=2, levels=3, precision=1),
}


# the shortest filters (Haar and db2, lengths 2 and 4) through one streamed pass: the vector
# windows of the row analysis and synthesis at their narrowest (Haar leaves the synthesis
# window's first vector unused)
SHORT = {
    "one-pass-128-haar": lambda: configs.small_lgs_config(n_sub=40, N=128, n_layers=2, levels=3, order=1),
    "one-pass-128-db2": lambda: configs.small_lgs_config(n_sub=40, N=128, n_layers=2, levels=3, order=2),
}


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


@pytest.fixture(scope="module", params=list(CASES))
def case(request, lib):
    torch, pkg = lib
    g = CASES[request.param]()
    plan = pkg.Plan(g, transforms=2)
    assert plan.info.streamed == 1 and plan.info.gather_separate == 1
    ora = Tomography(g)
    dt = torch.float64 if g["precision"] else torch.float32
    yield torch, pkg, g, plan, ora, dt, request.param
    plan.close()


def _tol(g, fp32):
    return 1e-11 if g["precision"] else fp32


def test_streamed_transforms(case):
    torch, pkg, g, plan, ora, dt, name = case
    rng = np.random.default_rng(21)
    c = rng.standard_normal(plan.n)
    out = torch.full((plan.n,), float("nan"), dtype=dt, device="cuda")
    plan.coeffs_to_layers(torch.tensor(c, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.join(ora.synthesis(c)), f"streamed-synthesis/{name}")
    assert e < _tol(g, 2e-6), e
    phi = rng.standard_normal(plan.n)
    plan.layers_to_coeffs(torch.tensor(phi, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.analysis(ora.split(phi)), f"streamed-analysis/{name}")
    assert e < _tol(g, 2e-6), e


def test_streamed_operator_and_rhs(case):
    torch, pkg, g, plan, ora, dt, name = case
    rng = np.random.default_rng(22)
    c = rng.standard_normal(plan.n)
    out = torch.full((plan.n,), float("nan"), dtype=dt, device="cuda")
    plan.apply_normal(torch.tensor(c, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.apply_normal(c), f"streamed-normal/{name}")
    assert e < _tol(g, 1e-5), e
    s = rng.standard_normal(plan.n_slopes)
    plan.rhs(torch.tensor(s, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.rhs(s), f"streamed-rhs/{name}")
    assert e < _tol(g, 1e-5), e


@pytest.mark.parametrize("warm", [False, True])
def test_streamed_solve(case, warm):
    torch, pkg, g, plan, ora, dt, name = case
    phis = FrozenFlow(g, 5).layers(0.002)
    s = ora.measure(phis) + gaussian_noise(plan.n_slopes, 0.1, 1_000_023)
    x0 = np.random.default_rng(23).standard_normal(plan.n) * 0.5 if warm else np.zeros(plan.n)
    iters = int(g["iters"])
    x_ref = ora.pcg(ora.rhs(s), x0, iters, ora.jacobi_diagonal())
    x = torch.tensor(x0, dtype=dt, device="cuda")
    resn = plan.solve(torch.tensor(s, dtype=dt, device="cuda"), x, iters, warm=warm, resnorm=True)
    e = rel(x.double().cpu().numpy(), x_ref, f"streamed-solve-{'warm' if warm else 'cold'}/{name}")
    assert e < _tol(g, 1e-5), e
    assert np.isfinite(resn) and resn > 0


def test_streamed_graph_equals_direct_launches(case):
    torch, pkg, g, plan, ora, dt, name = case
    rng = np.random.default_rng(24)
    s = torch.tensor(rng.standard_normal(plan.n_slopes), dtype=dt, device="cuda")
    x0 = torch.tensor(rng.standard_normal(plan.n), dtype=dt, device="cuda")
    outs = []
    for mode in (1, 0):
        plan.set_launch_mode(mode)
        x = x0.clone()
        plan.solve(s, x, 3, warm=True)
        outs.append(x)
    plan.set_launch_mode(1)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


def test_streamed_batch_is_bitwise_single_and_close_to_clusters(lib):
    torch, pkg = lib
    geoms = [CASES["one-pass-128"](), CASES["coarse-only-32"](), CASES["two-pass-256-db4"]()]
    plans = [pkg.Plan(g, transforms=2) for g in geoms]
    rng = np.random.default_rng(25)
    s = [torch.tensor(rng.standard_normal(p.n_slopes), dtype=torch.float32, device="cuda") for p in plans]
    x0 = [torch.tensor(rng.standard_normal(p.n), dtype=torch.float32, device="cuda") for p in plans]
    single = []
    for p, si, xi in zip(plans, s, x0):
        x = xi.clone()
        p.solve(si, x, 4, warm=True)
        single.append(x)
    xb = [xi.clone() for xi in x0]
    pkg.solve_batch(plans, s, xb, 4, warm=True)
    torch.cuda.synchronize()
    for a, b in zip(single, xb):
        assert torch.equal(a, b)
    # the cluster transforms of the same plans reach the same iterate up to rounding
    for g, p, si, xi, xs in zip(geoms, plans, s, x0, single):
        pc = pkg.Plan(g, transforms=1)
        assert pc.info.streamed == 0
        x = xi.clone()
        pc.solve(si, x, 4, warm=True)
        torch.cuda.synchronize()
        e = rel(xs.double().cpu().numpy(), x.double().cpu().numpy(), f"streamed-vs-cluster/{g['name']}")
        assert e < 1e-5, (g["name"], e)
        pc.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("name", list(SHORT))
def test_streamed_short_filters(lib, name):
    """Haar and db2 through the streamed passes: W, W^-1, the normal operator and the
    right-hand side against the FP64 oracle, and a three-iteration cold solve."""
    torch, pkg = lib
    g = SHORT[name]()
    plan = pkg.Plan(g, transforms=2)
    assert plan.info.streamed == 1 and plan.info.gather_separate == 1
    ora = Tomography(g)
    dt = torch.float32
    rng = np.random.default_rng(28)
    c = rng.standard_normal(plan.n)
    out = torch.full((plan.n,), float("nan"), dtype=dt, device="cuda")
    plan.coeffs_to_layers(torch.tensor(c, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.join(ora.synthesis(c)), f"streamed-synthesis/{name}")
    assert e < 2e-6, e
    plan.layers_to_coeffs(torch.tensor(c, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.analysis(ora.split(c)), f"streamed-analysis/{name}")
    assert e < 2e-6, e
    plan.apply_normal(torch.tensor(c, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.apply_normal(c), f"streamed-normal/{name}")
    assert e < 1e-5, e
    s = rng.standard_normal(plan.n_slopes)
    plan.rhs(torch.tensor(s, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.rhs(s), f"streamed-rhs/{name}")
    assert e < 1e-5, e
    phis = FrozenFlow(g, 5).layers(0.002)
    sl = ora.measure(phis) + gaussian_noise(plan.n_slopes, 0.1, 1_000_029)
    x_ref = ora.pcg(ora.rhs(sl), np.zeros(plan.n), 3, ora.jacobi_diagonal())
    x = torch.zeros(plan.n, dtype=dt, device="cuda")
    plan.solve(torch.tensor(sl, dtype=dt, device="cuda"), x, 3, warm=False)
    e = rel(x.double().cpu().numpy(), x_ref, f"streamed-solve-3it/{name}")
    assert e < 1e-5, e
    plan.close()


@pytest.mark.parametrize("name", ["eelt", "one-pass-128", "elongated-32", "one-pass-128-fp64"] + list(SHORT))
def test_cluster_and_streamed_paths_are_bitwise_the_same(lib, name):
    """Two independent implementations of every operator: thread-block clusters
    with the gather fused into the analysis (tables staged in shared memory), and
    streamed row-tile passes with the separate gather kernel.  They take every
    output's sums in the same order, so W, W^-1, the normal operator and the
    right-hand side agree bit for bit, FP32 and FP64, with elongated spots."""
    torch, pkg = lib
    g = {"eelt": configs.config1,
         "one-pass-128": CASES["one-pass-128"],
         "elongated-32": lambda: configs.with_elongation(configs.small_lgs_config(16, 32, 3, 2),
                                                         spot_fwhm_arcsec=0.5),
         "one-pass-128-fp64": CASES["one-pass-128-fp64"], **SHORT}[name]()
    dt = torch.float64 if g["precision"] else torch.float32
    outs = []
    for tf in (1, 2):
        p = pkg.Plan(g, transforms=tf)
        assert (p.info.streamed, p.info.gather_separate) == ((0, 0) if tf == 1 else (1, 1))
        rng = np.random.default_rng(27)
        c = torch.tensor(rng.standard_normal(p.n), dtype=dt, device="cuda")
        s = torch.tensor(rng.standard_normal(p.n_slopes), dtype=dt, device="cuda")
        res = [torch.empty(p.n, dtype=dt, device="cuda") for _ in range(4)]
        p.coeffs_to_layers(c, res[0])
        p.layers_to_coeffs(c, res[1])
        p.apply_normal(c, res[2])
        p.rhs(s, res[3])
        torch.cuda.synchronize()
        outs.append(res)
        p.close()
    for what, a, b in zip(("synthesis", "analysis", "normal", "rhs"), outs[0], outs[1]):
        assert torch.equal(a, b), what
