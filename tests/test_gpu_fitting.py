"""The fitting step on the GPU (Sec. 4.1, eqs. fit_step_ideal / fit_step_min)
against the FP64 oracle: the normal operator H^T H, the right-hand side
H^T P phi and CG solves (cold and warm), on a small system, a system whose
mirror grids are cut by the field (taps outside the grid) with wide actuator
windows, and the E-ELT system with the paper's three mirrors and 5 x 5
directions; tomo_reconstruct against the same steps called one by one."""
import numpy as np
import pytest

from oracle import Fitting, Tomography
from synth import configs, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu


def _small(precision=0):
    g = configs.small_lgs_config(16, 32, 3, 2, precision=precision)
    return configs.with_fitting(g, altitudes=(0.0, 4000.0, 9000.0), pitches=(0.5, 0.72, 1.0),
                                field_arcmin=1.2, n_dir=3)


def _cut():
    """Mirrors narrower than the footprints (points beyond the outermost actuators)
    and pitches up to 4 subapertures (8-corner windows)."""
    g = configs.with_fitting(configs.small_lgs_config(16, 32, 3, 2), altitudes=(0.0, 6000.0),
                             pitches=(1.25, 2.0), field_arcmin=1.2, n_dir=4)
    g["fitting"]["dms"][0]["n"] = 5
    g["fitting"]["dms"][1]["n"] = 7
    return g


def _single():
    """The degenerate case: one mirror seen from one direction (on axis)."""
    return configs.with_fitting(configs.small_lgs_config(16, 32, 3, 2), altitudes=(0.0,), pitches=(0.5,),
                                field_arcmin=0.0, n_dir=1)


CASES = {
    "small": _small,
    "single-mirror-single-direction": _single,
    "small-fp64": lambda: _small(1),
    "cut-mirrors": _cut,
    "eelt": lambda: configs.with_fitting(configs.config1()),
}


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


@pytest.mark.parametrize("name", list(CASES))
def test_fitting_operator_rhs_and_solve(lib, name):
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    ora = Fitting(g)
    tom = Tomography(g)
    assert fit.n == ora.n
    assert fit.info.n_active == ora.active_actuators()
    assert fit.info.n_points == ora.n_points
    dt = plan.dtype
    tol = 1e-11 if g["precision"] else 1e-5
    rng = np.random.default_rng(11)
    a = rng.standard_normal(ora.n)
    out = torch.empty(ora.n, dtype=dt, device="cuda")
    fit.apply_normal(torch.tensor(a, dtype=dt, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.apply_normal(a), f"fit-normal/{name}")
    assert e < tol, e
    phis = tom.synthesis(rng.standard_normal(tom.n))
    layers = torch.tensor(tom.join(phis), dtype=dt, device="cuda")
    b = torch.empty(ora.n, dtype=dt, device="cuda")
    fit.rhs(layers, b)
    b_ref = ora.rhs(phis)
    e = rel(b.double().cpu().numpy(), b_ref, f"fit-rhs/{name}")
    assert e < tol, e
    # cold start, the paper's 4 iterations
    x = torch.full((ora.n,), float("nan"), dtype=dt, device="cuda")
    fit.solve(layers, x, 4, warm=False)
    x_ref = ora.cg(b_ref, np.zeros(ora.n), 4)
    e = rel(x.double().cpu().numpy(), x_ref, f"fit-solve-cold/{name}")
    assert e < tol, e
    # warm start from a perturbed solution
    x0 = x_ref + 0.1 * rng.standard_normal(ora.n)
    x = torch.tensor(x0, dtype=dt, device="cuda")
    fit.solve(layers, x, 4, warm=True)
    e = rel(x.double().cpu().numpy(), ora.cg(b_ref, x0, 4), f"fit-solve-warm/{name}")
    assert e < tol, e
    fit.close()
    plan.close()


def test_fitting_solve_is_deterministic_and_zero_iterations_give_zero(lib):
    torch, pkg = lib
    g = _small()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    layers = torch.tensor(np.random.default_rng(12).standard_normal(plan.n), dtype=torch.float32, device="cuda")
    xs = []
    for _ in range(2):
        x = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
        fit.solve(layers, x, 6, warm=False)
        xs.append(x)
    assert torch.equal(xs[0], xs[1])
    z = torch.full((fit.n,), 7.0, dtype=torch.float32, device="cuda")
    fit.solve(layers, z, 0, warm=False)
    assert torch.count_nonzero(z).item() == 0
    fit.close()
    plan.close()


@pytest.mark.parametrize("name", ["small", "eelt"])
def test_reconstruct_is_the_steps_one_by_one(lib, name):
    """tomo_reconstruct (one graph) == tomo_solve, then W^-1, then tomo_fit_solve;
    and the chain matches the oracle's tomography solve followed by its fitting."""
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    tom = Tomography(g)
    ora = Fitting(g)
    s = tom.measure(tom.synthesis(np.random.default_rng(13).standard_normal(tom.n))) + \
        gaussian_noise(plan.n_slopes, 0.3, 14)
    ds = torch.tensor(s, dtype=torch.float32, device="cuda")
    iters, fit_iters = 6, 4
    # one by one
    c1 = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
    a1 = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
    lay = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    plan.solve(ds, c1, iters, warm=False)
    plan.coeffs_to_layers(c1, lay)
    fit.solve(lay, a1, fit_iters, warm=False)
    # fused, twice (graph capture, then replay)
    for _ in range(2):
        c2 = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
        a2 = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
        fit.reconstruct(ds, c2, a2, iters, fit_iters, warm=False)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2) and torch.equal(a1, a2)
    c_ref = tom.solve(s, np.zeros(tom.n), iters)
    a_ref = ora.solve(tom.synthesis(c_ref), np.zeros(ora.n), fit_iters)
    e = rel(a2.double().cpu().numpy(), a_ref, f"reconstruct/{name}")
    assert e < 1e-5, e
    fit.close()
    plan.close()


def test_fitting_rejects_bad_geometry(lib):
    torch, pkg = lib
    g = _small()
    plan = pkg.Plan(g)
    bad = dict(g["fitting"], dms=[dict(g["fitting"]["dms"][0], pitch=3.0)])   # pitch > 4 d_sub
    with pytest.raises(pkg.TomoError) as ei:
        pkg.Fit(plan, bad)
    assert ei.value.status == 1
    empty = dict(g["fitting"], valid=np.zeros_like(g["fitting"]["valid"]))
    with pytest.raises(pkg.TomoError) as ei:
        pkg.Fit(plan, empty)
    assert ei.value.status == 2
    # a 2x2 sampling grid (3 corners per side) under 1 m actuators: 3-corner windows, which the
    # gather rounds up to 4 taps, more than the grid holds
    tiny = dict(g["fitting"], n_sub=2, valid=np.ones((2, 2), np.uint8),
                dms=[{"altitude": 0.0, "pitch": 1.0, "n": 5}])
    with pytest.raises(pkg.TomoError) as ei:
        pkg.Fit(plan, tiny)
    assert ei.value.status == 8
    plan.close()


@pytest.mark.parametrize("name", ["small", "small-fp64", "eelt"])
def test_residual_rms_per_direction(lib, name):
    """The quality measure of Sec. 5.1: per-direction piston-removed RMS of the
    residual wavefront, with and without a correction, against the oracle."""
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    tom, ora = Tomography(g), Fitting(g)
    dt = plan.dtype
    tol = 1e-11 if g["precision"] else 1e-5
    rng = np.random.default_rng(15)
    phis = tom.synthesis(rng.standard_normal(tom.n))
    layers = torch.tensor(tom.join(phis), dtype=dt, device="cuda")
    a = ora.solve(phis, np.zeros(ora.n), 4)
    out = torch.empty(len(ora.theta), dtype=torch.float64, device="cuda")
    for cmd in (None, a):
        fit.residual_rms(layers, None if cmd is None else torch.tensor(cmd, dtype=dt, device="cuda"), out)
        want = ora.residual_rms(phis, np.zeros(ora.n) if cmd is None else cmd)
        e = rel(out.cpu().numpy(), want, f"fit-rms/{name}/{'open' if cmd is None else 'fitted'}")
        assert e < tol, e
    fit.close()
    plan.close()


@pytest.mark.parametrize("name", ["single-mirror-single-direction", "cut-mirrors"])
def test_normal_matrix_entries_match_the_brute_force_pattern(lib, name):
    """The stored entries of H^T H are the actuator pairs that share a sampling
    point with nonzero weights in some direction (all weights are positive, so no
    sum cancels).  Pairs whose weight product is a rounding residue sit on a hat's
    edge, where the two sides may decide either way: the count lies between the
    pattern with those dropped and the full pattern."""
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    H = Fitting(g).dense_mirror_bruteforce()
    hi = int(np.count_nonzero((H != 0).T.astype(np.int64) @ (H != 0).astype(np.int64)))
    big = np.abs(H) > 1e-9
    lo = int(np.count_nonzero(big.T.astype(np.int64) @ big.astype(np.int64)))
    assert lo <= fit.info.normal_nonzeros <= hi, (lo, fit.info.normal_nonzeros, hi)
    assert fit.info.bytes_per_iteration > fit.info.normal_nonzeros * (8 if g["precision"] else 4)
    fit.close()
    plan.close()


def test_solve_that_converges_in_one_iteration_stays_put(lib):
    """One mirror on the sampling points, seen from one direction: H^T H is the
    identity on the reached actuators, so CG is exact after one iteration.  The
    later iterations must leave the commands where they are (r = 0 gives
    alpha = 0), however many are asked for."""
    torch, pkg = lib
    g = _single()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    ora = Fitting(g)
    tom = Tomography(g)
    phis = tom.synthesis(np.random.default_rng(19).standard_normal(tom.n))
    layers = torch.tensor(tom.join(phis), dtype=plan.dtype, device="cuda")
    b_ref = ora.rhs(phis)
    for iters in (1, 2, 12):
        x = torch.full((ora.n,), float("nan"), dtype=plan.dtype, device="cuda")
        fit.solve(layers, x, iters, warm=False)
        e = rel(x.double().cpu().numpy(), ora.cg(b_ref, np.zeros(ora.n), iters), f"fit-exact-iterate/{iters}")
        assert e < 1e-5, (iters, e)
    fit.close()
    plan.close()
