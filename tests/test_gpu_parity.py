"""GPU parity: every operator of the solve and the full fixed-iteration (P)CG
frame, through the C ABI, against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 over the whole output):
* FP32 operator (precision 0): transforms 2e-6, measurement/normal operator/
  right-hand side 1e-5 (Fried differences of nearby phase values cancel), the
  solve 1e-5 on the reconstructed layers (the target of the method), the
  Jacobi diagonal 1e-12 (computed in FP64 on the device);
* FP64 operator (precision 1): 1e-11 everywhere.
"""
import json
import os

import numpy as np
import pytest

from oracle import Tomography
from synth import configs, FrozenFlow, gaussian_noise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    return torch


ERRORS = {}


@pytest.fixture(scope="module", autouse=True)
def error_log():
    """Measured errors, written to $TOMO_PARITY_LOG (JSON) when it is set."""
    yield
    path = os.environ.get("TOMO_PARITY_LOG")
    if path:
        old = json.load(open(path)) if os.path.exists(path) else {}
        old.update(ERRORS)
        json.dump(old, open(path, "w"), indent=1, sort_keys=True)


def rel(a, b, key=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    e = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    if key is not None:
        ERRORS[key] = e
    return e


def tol(geom, fp32):
    return 1e-11 if geom["precision"] == 1 else fp32


CASES = {
    "small-lgs": lambda: configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2),
    "ragged-multitile": lambda: configs.small_lgs_config(n_sub=40, N=64, n_layers=4, levels=3),
    "wrap": lambda: configs.small_lgs_config(n_sub=12, N=32, n_layers=3, levels=2, wrap=True),
    "db4-J1": lambda: configs.small_lgs_config(n_sub=16, N=32, n_layers=2, levels=1, order=4),
    # The worst-conditioned case of the set (Haar, three levels on 16^2: the
    # Jacobi-preconditioned normal matrix has condition number 7.5e5), at its
    # configuration's 8 PCG iterations.  CG amplifies the rounding of every
    # operator application steeply with the iteration count here: the FP32 path
    # measured 1.1e-7, 8.2e-7, 3.8e-6 after 1, 4, 8 iterations and 2.3e-5, 4.3e-4
    # after 9, 10 (the FP64 path 2e-16 ... 4e-13 over the same counts), and an
    # FP64 emulation that only rounds the operator's and the state's values to
    # FP32 gives 2e-6 at 8 and 2e-4 at 10: the growth is the problem's, not the
    # kernels'.
    "haar-N16": lambda: configs.small_lgs_config(n_sub=8, N=16, n_layers=2, levels=3, order=1,
                                                 d_sub=0.5, dx=0.5),
    "db2-noprecond": lambda: configs.small_lgs_config(n_sub=16, N=32, n_layers=2, levels=3,
                                                      order=2, precond=0),
    "small-fp64": lambda: configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2,
                                                   precision=1),
    "cfg0-fp64": configs.config0,
}


class Case:
    def __init__(self, torch, geom):
        import paper_1302_3734_gb300 as pkg
        self.torch = torch
        self.geom = geom
        self.ora = Tomography(geom)
        self.plan = pkg.Plan(geom)
        self.dt = torch.float64 if geom["precision"] else torch.float32
        assert self.plan.n == self.ora.n and self.plan.n_slopes == self.ora.meas_offsets[-1]

    def dev(self, x):
        return self.torch.tensor(np.asarray(x), dtype=self.dt, device="cuda")

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.double().cpu().numpy()

    def empty(self, n):
        return self.torch.full((n,), float("nan"), dtype=self.dt, device="cuda")


@pytest.fixture(scope="module", params=list(CASES))
def case(request, torch_cuda):
    c = Case(torch_cuda, CASES[request.param]())
    yield c
    c.plan.close()


def test_synthesis(case):
    c = np.random.default_rng(1).standard_normal(case.ora.n)
    out = case.empty(case.ora.n)
    case.plan.coeffs_to_layers(case.dev(c), out)
    assert rel(case.host(out), case.ora.join(case.ora.synthesis(c)),
               f"synthesis/{case.geom['name']}") < tol(case.geom, 2e-6)


def test_analysis(case):
    phi = np.random.default_rng(2).standard_normal(case.ora.n)
    out = case.empty(case.ora.n)
    case.plan.layers_to_coeffs(case.dev(phi), out)
    assert rel(case.host(out), case.ora.analysis(case.ora.split(phi)),
               f"analysis/{case.geom['name']}") < tol(case.geom, 2e-6)


def test_measurement(case):
    phis = FrozenFlow(case.geom, 3).layers(0.0)
    out = case.empty(case.plan.n_slopes)
    case.plan.layers_to_slopes(case.dev(case.ora.join(phis)), out)
    assert rel(case.host(out), case.ora.measure(phis),
               f"measurement/{case.geom['name']}") < tol(case.geom, 1e-5)


def test_normal_operator(case):
    c = np.random.default_rng(3).standard_normal(case.ora.n)
    out = case.empty(case.ora.n)
    case.plan.apply_normal(case.dev(c), out)
    assert rel(case.host(out), case.ora.apply_normal(c),
               f"normal/{case.geom['name']}") < tol(case.geom, 1e-5)


def test_rhs(case):
    s = np.random.default_rng(4).standard_normal(case.plan.n_slopes)
    out = case.empty(case.ora.n)
    case.plan.rhs(case.dev(s), out)
    assert rel(case.host(out), case.ora.rhs(s), f"rhs/{case.geom['name']}") < tol(case.geom, 1e-5)


def test_jacobi_diagonal(case):
    out = case.torch.empty(case.ora.n, dtype=case.torch.float64, device="cuda")
    case.plan.jacobi_diagonal(out)
    assert rel(case.host(out), case.ora.jacobi_diagonal(), f"jacobi/{case.geom['name']}") < 1e-12
    if case.ora.n <= 3072:
        # and against the diagonal's definition, one unit vector at a time (not the
        # oracle's separable-profile route, whose idea the kernel shares)
        assert rel(case.host(out), case.ora.jacobi_diagonal_probe(), f"jacobi-def/{case.geom['name']}") < 1e-12


def _frame(case, seed=7):
    phis = FrozenFlow(case.geom, 5).layers(0.002)
    s = case.ora.measure(phis) + gaussian_noise(case.plan.n_slopes, 0.1, 1_000_000 + seed)
    x0 = np.random.default_rng(seed).standard_normal(case.ora.n) * 0.5
    return s, x0


@pytest.mark.parametrize("warm", [False, True])
def test_solve(case, warm):
    s, x0 = _frame(case)
    iters = int(case.geom["iters"])
    pre = case.ora.jacobi_diagonal() if case.geom["precond"] else None
    x_ref = case.ora.pcg(case.ora.rhs(s), x0 if warm else np.zeros(case.ora.n), iters, pre)
    coeffs = case.dev(x0) if warm else case.empty(case.ora.n)
    resn = case.plan.solve(case.dev(s), coeffs, iters, warm=warm, resnorm=True)
    x = case.host(coeffs)
    phi = case.ora.join(case.ora.synthesis(x))
    phi_ref = case.ora.join(case.ora.synthesis(x_ref))
    assert rel(phi, phi_ref, f"solve-{'warm' if warm else 'cold'}/{case.geom['name']}") < tol(case.geom, 1e-5)
    assert np.isfinite(resn) and resn > 0


def test_zero_iterations(case):
    s, x0 = _frame(case)
    coeffs = case.dev(x0)
    case.plan.solve(case.dev(s), coeffs, 0, warm=True)
    assert rel(case.host(coeffs), x0) < 1e-7
    coeffs = case.empty(case.ora.n)
    case.plan.solve(case.dev(s), coeffs, 0, warm=False)
    assert np.all(case.host(coeffs) == 0.0)


def test_deterministic_and_graph_equals_direct(case):
    s, x0 = _frame(case, seed=11)
    outs = []
    for mode in (1, 1, 0):
        case.plan.set_launch_mode(mode)
        coeffs = case.dev(x0)
        case.plan.solve(case.dev(s), coeffs, 3, warm=True)
        outs.append(case.host(coeffs))
    case.plan.set_launch_mode(1)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_nan_data_reports_breakdown(torch_cuda):
    import paper_1302_3734_gb300 as pkg
    g = configs.small_lgs_config(n_sub=8, N=32, n_layers=2, levels=2)
    plan = pkg.Plan(g)
    s = torch_cuda.full((plan.n_slopes,), float("nan"), device="cuda")
    x = torch_cuda.zeros(plan.n, device="cuda")
    with pytest.raises(pkg.TomoError) as e:
        plan.solve(s, x, 3, warm=False, resnorm=True)
    assert e.value.status == 7
    # the plan stays usable after a breakdown
    s.zero_()
    assert plan.solve(s, x, 2, warm=False, resnorm=True) == 0.0
    plan.close()


def test_breakdown_without_resnorm_is_reported_by_the_next_call(torch_cuda):
    """NaN slopes in a graph-replayed solve without out_resnorm: the iterate stays
    x0 (frozen), the plan's breakdown word is set, and the next tomo_solve returns
    TOMO_ERR_BREAKDOWN without enqueuing anything; the call after it solves."""
    import paper_1302_3734_gb300 as pkg
    g = configs.small_lgs_config(n_sub=8, N=32, n_layers=2, levels=2)
    plan = pkg.Plan(g)
    rng = np.random.default_rng(17)
    x0 = torch_cuda.tensor(rng.standard_normal(plan.n), dtype=torch_cuda.float32, device="cuda")
    good = torch_cuda.tensor(rng.standard_normal(plan.n_slopes), dtype=torch_cuda.float32, device="cuda")
    bad = torch_cuda.full((plan.n_slopes,), float("nan"), device="cuda")
    x = x0.clone()
    plan.solve(good, x, 3, warm=True)          # the graph of this signature exists
    torch_cuda.cuda.synchronize()
    assert plan._info().breakdown_pending == 0
    x.copy_(x0)
    plan.solve(bad, x, 3, warm=True)           # returns at once: no synchronisation
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(x, x0), "the iterate was not frozen at x0"
    assert plan._info().breakdown_pending == 1
    with pytest.raises(pkg.TomoError) as e:
        plan.solve(good, x, 3, warm=True)
    assert e.value.status == 7
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(x, x0), "the reporting call enqueued work"
    assert plan._info().breakdown_pending == 0
    plan.solve(good, x, 3, warm=True)
    ref = x0.clone()
    plan.set_launch_mode(0)
    plan.solve(good, ref, 3, warm=True)
    plan.set_launch_mode(1)
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(x, ref) and bool(torch_cuda.isfinite(x).all())
    plan.close()


def test_batch_breakdown_is_reported_by_the_next_batch_call(torch_cuda):
    """One instance of a batch gets NaN slopes: the other instance's result is its
    single solve, the broken one stays at x0, and the next tomo_solve_batch reports it."""
    import paper_1302_3734_gb300 as pkg
    geoms = [configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2),
             configs.small_lgs_config(n_sub=12, N=32, n_layers=2, levels=2)]
    plans = [pkg.Plan(g) for g in geoms]
    rng = np.random.default_rng(19)
    s = [torch_cuda.tensor(rng.standard_normal(p.n_slopes), dtype=torch_cuda.float32, device="cuda")
         for p in plans]
    x0 = [torch_cuda.tensor(rng.standard_normal(p.n), dtype=torch_cuda.float32, device="cuda")
          for p in plans]
    alone = x0[0].clone()
    plans[0].solve(s[0], alone, 4, warm=True)
    bad = [s[0], torch_cuda.full_like(s[1], float("nan"))]
    xb = [xi.clone() for xi in x0]
    pkg.solve_batch(plans, bad, xb, 4, warm=True)
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(xb[0], alone) and torch_cuda.equal(xb[1], x0[1])
    assert [p._info().breakdown_pending for p in plans] == [0, 1]
    with pytest.raises(pkg.TomoError) as e:
        pkg.solve_batch(plans, s, xb, 4, warm=True)
    assert e.value.status == 7
    assert [p._info().breakdown_pending for p in plans] == [0, 0]
    pkg.solve_batch(plans, s, xb, 4, warm=True)
    torch_cuda.cuda.synchronize()
    assert all(bool(torch_cuda.isfinite(x).all()) for x in xb)
    for p in plans:
        p.close()


def test_zero_data_cold_start_is_exact(torch_cuda):
    import paper_1302_3734_gb300 as pkg
    g = configs.small_lgs_config(n_sub=8, N=32, n_layers=2, levels=2)
    plan = pkg.Plan(g)
    s = torch_cuda.zeros(plan.n_slopes, device="cuda")
    x = torch_cuda.full((plan.n,), 5.0, device="cuda")
    assert plan.solve(s, x, 4, warm=False, resnorm=True) == 0.0
    torch_cuda.cuda.synchronize()
    assert float(x.abs().max()) == 0.0
    plan.close()


def test_batch_equals_single(torch_cuda):
    import paper_1302_3734_gb300 as pkg
    geoms = [configs.small_lgs_config(n_sub=16, N=32, n_layers=3, levels=2),
             configs.small_lgs_config(n_sub=12, N=32, n_layers=2, levels=2)]
    plans = [pkg.Plan(g) for g in geoms]
    rng = np.random.default_rng(5)
    s = [torch_cuda.tensor(rng.standard_normal(p.n_slopes), dtype=torch_cuda.float32, device="cuda")
         for p in plans]
    x0 = [torch_cuda.tensor(rng.standard_normal(p.n), dtype=torch_cuda.float32, device="cuda")
          for p in plans]
    single = []
    for p, si, xi in zip(plans, s, x0):
        x = xi.clone()
        p.solve(si, x, 5, warm=True)
        single.append(x)
    xb = [xi.clone() for xi in x0]
    pkg.solve_batch(plans, s, xb, 5, warm=True)
    torch_cuda.cuda.synchronize()
    for a, b in zip(single, xb):
        assert torch_cuda.equal(a, b)
    for p in plans:
        p.close()
