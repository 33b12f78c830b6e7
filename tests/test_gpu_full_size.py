"""Full-size parity at the E-ELT workload the benchmark times (84x84 LGS
sensors, 9 layers of 128^2, db3 J=4, 10 Jacobi-PCG iterations, warm start),
in the benchmark's launch configuration (CUDA-graph replay).

Each frame of a short frozen-flow sequence is solved on the GPU; the oracle
solves the same frame from the same x0 (the GPU's previous result, widened to
FP64), so every comparison measures one solve, not accumulated drift.
"""
import numpy as np
import pytest

from oracle import Tomography
from synth import configs, FrozenFlow, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    g = configs.config1()
    ora = Tomography(g)
    plan = pkg.Plan(g)
    yield torch, g, ora, plan
    plan.close()


def test_jacobi_diagonal_full_size(setup):
    torch, g, ora, plan = setup
    out = torch.empty(plan.n, dtype=torch.float64, device="cuda")
    plan.jacobi_diagonal(out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ora.jacobi_diagonal(), "jacobi/full-size") < 1e-12


def test_normal_operator_full_size(setup):
    torch, g, ora, plan = setup
    c = np.random.default_rng(31).standard_normal(plan.n)
    out = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    plan.apply_normal(torch.tensor(c, dtype=torch.float32, device="cuda"), out)
    torch.cuda.synchronize()
    assert rel(out.double().cpu().numpy(), ora.apply_normal(c), "normal/full-size") < 1e-5


def test_frame_sequence_full_size(setup):
    torch, g, ora, plan = setup
    ff = FrozenFlow(g, 1)
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in g["wfs"]])
    Jd = ora.jacobi_diagonal()
    x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
    plan.set_launch_mode(1)
    for k in range(3):
        s = ora.measure(ff.layers(0.002 * k)) + gaussian_noise(plan.n_slopes, 1.0, 5_000 + k) * sig
        x0 = x.double().cpu().numpy()
        warm = k > 0
        plan.solve(torch.tensor(s, dtype=torch.float32, device="cuda"), x, g["iters"], warm=warm)
        torch.cuda.synchronize()
        x_ref = ora.pcg(ora.rhs(s), x0 if warm else np.zeros(plan.n), g["iters"], Jd)
        phi = ora.join(ora.synthesis(x.double().cpu().numpy()))
        phi_ref = ora.join(ora.synthesis(x_ref))
        assert rel(phi, phi_ref, f"solve-frame{k}/full-size") < 1e-5, k
