"""Plans at every allowed cluster size (CTAs per layer in the transform kernels,
the launch shape the autotuner picks) compute the same operator and solve as
the FP64 oracle, and the autotuner returns a measured, buildable size."""
import numpy as np
import pytest

from oracle import Tomography
from synth import configs, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu

GEOMS = {
    "small-32": configs.small_lgs_config(16, 32, 3, 2),
    "ragged-64": configs.small_lgs_config(24, 64, 2, 3, order=2),
}


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_operator_and_solve_at_cluster_size(lib, name, C):
    torch, pkg = lib
    g = GEOMS[name]
    if C > min(l["N"] for l in g["layers"]) // 2:
        pytest.skip("cluster size above N/2")
    plan = pkg.Plan(g, cluster_size=C)
    assert plan.info.cluster_size == C
    ora = Tomography(g)
    rng = np.random.default_rng(C)
    x = rng.standard_normal(plan.n)
    out = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    plan.apply_normal(torch.tensor(x, dtype=torch.float32, device="cuda"), out)
    e = rel(out.double().cpu().numpy(), ora.apply_normal(x), f"normal-C{C}/{name}")
    assert e < 1e-5, e
    s = gaussian_noise(plan.n_slopes, 0.5, 11 + C)
    xs = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
    plan.solve(torch.tensor(s, dtype=torch.float32, device="cuda"), xs, 6, warm=False)
    x_ref = ora.pcg(ora.rhs(s), np.zeros(ora.n), 6, ora.jacobi_diagonal())
    e = rel(ora.join(ora.synthesis(xs.double().cpu().numpy())), ora.join(ora.synthesis(x_ref)),
            f"solve-C{C}/{name}")
    assert e < 1e-5, e
    plan.close()


def test_autotuner_picks_a_measured_buildable_size(lib, tmp_path):
    torch, pkg = lib
    from paper_1302_3734_gb300 import autotune
    geoms = [GEOMS["small-32"], GEOMS["ragged-64"], GEOMS["small-32"]]
    path = str(tmp_path / "tune.json")
    best, table = autotune.tune_cluster_size(geoms, iters=4, candidates=(8, 4, 2), steps=3, path=path)
    assert best in (8, 4, 2) and table[best] == max(v for v in table.values() if v)
    # cached: the second call returns the same choice without measuring
    assert autotune.tune_cluster_size(geoms, iters=4, candidates=(8, 4, 2), path=path)[0] == best
    plans = autotune._plans(geoms, best)
    assert all(p.info.cluster_size >= best for p in plans)
    for p in plans:
        p.close()
