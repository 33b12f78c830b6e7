"""Pseudo-open-loop control on the GPU (Sec. 4.2, Algorithm 4.1) against the FP64
oracle: the mirrors measured by the sensors (A_hat), one control step, and a
closed loop over a frozen-flow atmosphere in which each side closes its own
loop (residual data = measurement - A_hat a_{t-2})."""
import numpy as np
import pytest

from oracle.control import Control
from synth import configs, FrozenFlow, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu


def _small(precision=0):
    g = configs.small_lgs_config(16, 32, 3, 2, precision=precision)
    return configs.with_fitting(g, altitudes=(0.0, 4000.0, 9000.0), pitches=(0.5, 0.72, 1.0),
                                field_arcmin=1.2, n_dir=3)


CASES = {
    "small": _small,
    "small-fp64": lambda: _small(1),
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
def test_mirror_slopes(lib, name):
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    ctl = Control(g)
    dt = plan.dtype
    tol = 1e-11 if g["precision"] else 1e-5
    rng = np.random.default_rng(31)
    a = rng.standard_normal(fit.n)
    base = rng.standard_normal(plan.n_slopes)
    out = torch.empty(plan.n_slopes, dtype=dt, device="cuda")
    fit.mirror_slopes(torch.tensor(a, dtype=dt, device="cuda"), out)
    want = ctl.mirror_slopes(a)
    e = rel(out.double().cpu().numpy(), want, f"mirror-slopes/{name}")
    assert e < tol, e
    # in-place residual form: out = base - A_hat a
    sl = torch.tensor(base, dtype=dt, device="cuda")
    fit.mirror_slopes(torch.tensor(a, dtype=dt, device="cuda"), sl, slopes_in=sl, scale=-1.0)
    e = rel(sl.double().cpu().numpy(), base - want, f"mirror-slopes-residual/{name}")
    assert e < tol, e
    fit.close()
    plan.close()


@pytest.mark.parametrize("name", ["small", "small-fp64", "eelt"])
def test_control_step(lib, name):
    torch, pkg = lib
    g = CASES[name]()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    ctl = Control(g)
    dt = plan.dtype
    tol = 1e-9 if g["precision"] else 1e-5
    rng = np.random.default_rng(32)
    tom = ctl.tom
    s = tom.measure(tom.synthesis(rng.standard_normal(tom.n))) + gaussian_noise(plan.n_slopes, 0.3, 33)
    a_tm2, a_tm1 = 0.1 * rng.standard_normal(fit.n), 0.1 * rng.standard_normal(fit.n)
    x_prev = 0.1 * rng.standard_normal(tom.n)
    a_prev = 0.1 * rng.standard_normal(fit.n)
    T = lambda v: torch.tensor(v, dtype=dt, device="cuda")
    x, a_rec, a_t = T(x_prev), T(a_prev), torch.empty(fit.n, dtype=dt, device="cuda")
    fit.polc_step(T(s), x, a_rec, T(a_tm2), T(a_tm1), a_t, 0.4, 6, 4, warm=True)
    want_t, want_x, want_rec = ctl.step(s, a_tm2, a_tm1, x_prev, a_prev, 0.4, 6, 4)
    for got, want, what in ((x, want_x, "coeffs"), (a_rec, want_rec, "a_rec"), (a_t, want_t, "a_t")):
        e = rel(got.double().cpu().numpy(), want, f"polc-step/{name}/{what}")
        assert e < tol, (what, e)
    fit.close()
    plan.close()


def test_closed_loop_against_the_oracle_loop(lib):
    """Eight frames at 500 Hz of a frozen-flow atmosphere, gain 0.4, two-frame delay,
    warm starts; the GPU keeps two command buffers (a_t overwrites a_{t-2})."""
    torch, pkg = lib
    g = _small()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    ctl = Control(g)
    tom = ctl.tom
    flow = FrozenFlow(g, 3, instance=1)
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"]) for w in g["wfs"]])
    gain, iters, fit_iters, K = 0.4, 6, 4, 8
    # oracle loop
    a_o = [np.zeros(fit.n), np.zeros(fit.n)]
    x_o, rec_o = np.zeros(tom.n), np.zeros(fit.n)
    data = []
    for t in range(K):
        m = tom.measure(flow.layers(0.002 * t)) + gaussian_noise(plan.n_slopes, 1.0, 700 + t) * sig
        data.append(m)
        s = m - ctl.mirror_slopes(a_o[-2])
        a_t, x_o, rec_o = ctl.step(s, a_o[-2], a_o[-1], x_o, rec_o, gain, iters, fit_iters)
        a_o.append(a_t)
    # GPU loop
    buf = [torch.zeros(fit.n, dtype=torch.float32, device="cuda") for _ in range(2)]
    x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
    rec = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
    s = torch.empty(plan.n_slopes, dtype=torch.float32, device="cuda")
    for t in range(K):
        a_tm2, a_tm1 = buf[t % 2], buf[(t + 1) % 2]
        fit.mirror_slopes(a_tm2, s, slopes_in=torch.tensor(data[t], dtype=torch.float32, device="cuda"), scale=-1.0)
        fit.polc_step(s, x, rec, a_tm2, a_tm1, a_tm2, gain, iters, fit_iters, warm=t > 0)
        got = a_tm2.double().cpu().numpy()
        e = rel(got, a_o[t + 2], f"closed-loop/frame{t}")
        assert e < 1e-5, (t, e)
    fit.close()
    plan.close()


def test_control_step_graph_and_launch_mode_agree_bitwise(lib):
    torch, pkg = lib
    g = _small()
    out = []
    for graphs in (True, False):
        plan = pkg.Plan(g)
        plan.set_launch_mode(graphs)
        fit = pkg.Fit(plan, g["fitting"])
        rng = np.random.default_rng(34)
        T = lambda v: torch.tensor(v, dtype=torch.float32, device="cuda")
        s = T(rng.standard_normal(plan.n_slopes))
        a2, a1 = T(rng.standard_normal(fit.n)), T(rng.standard_normal(fit.n))
        x, rec, at = (torch.zeros(plan.n, device="cuda"), torch.zeros(fit.n, device="cuda"),
                      torch.zeros(fit.n, device="cuda"))
        for _ in range(2):
            fit.polc_step(s, x, rec, a2, a1, at, 0.4, 5, 4, warm=True)
        torch.cuda.synchronize()
        out.append((x.clone(), rec.clone(), at.clone()))
        fit.close()
        plan.close()
    for u, v in zip(out[0], out[1]):
        assert torch.equal(u, v)


def test_control_step_rejects_aliased_buffers(lib):
    torch, pkg = lib
    g = _small()
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    s = torch.zeros(plan.n_slopes, device="cuda")
    x = torch.zeros(plan.n, device="cuda")
    a = [torch.zeros(fit.n, device="cuda") for _ in range(3)]
    with pytest.raises(pkg.TomoError) as ei:
        fit.polc_step(s, x, a[0], a[1], a[2], a[2], 0.4, 2, 2)   # a_t == a_tm1
    assert ei.value.status == 1
    with pytest.raises(pkg.TomoError):
        fit.polc_step(s, x, a[1], a[1], a[2], a[0], 0.4, 2, 2)   # a_rec == a_tm2
    fit.close()
    plan.close()
