"""The regularisation-weight sweep of the quality metric through the GPU path,
point by point against the oracle (Sec. 5.2, the role of alpha; Sec. 5.1,
residual RMS): for every alpha of the sweep, tomo_reconstruct (30 PCG
iterations, W^-1, 4 fitting CG iterations) and tomo_fit_residual_rms against
the truth, compared with the oracle's reconstruction, commands and residual
RMS per direction; the GPU curve has its minimum at the same alpha.

Tolerances: the commands 1e-5 relative L2 (the FP32 path's target); the
residual RMS per direction 1e-5 relative (an RMS of FP32 fields of a few rad,
accumulated in double-float).
"""
import numpy as np
import pytest

import quality_sweep as qs
from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


def test_alpha_sweep_matches_the_oracle(lib):
    torch, pkg = lib
    frames = [qs.frame(k) for k in range(qs.FRAMES)]
    gpu_curve, ora_curve = {}, {}
    for alpha in qs.ALPHAS:
        g = qs.geometry(alpha)
        plan = pkg.Plan(g)
        fit = pkg.Fit(plan, g["fitting"])
        rms_g, rms_o = [], []
        for k, (truth, s) in enumerate(frames):
            _, a_ref, r_ref = qs.oracle_point(alpha, truth, s)
            x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
            a = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
            fit.reconstruct(torch.tensor(s, dtype=torch.float32, device="cuda"), x, a, qs.ITERS,
                            qs.FIT_ITERS, warm=False)
            truth_d = torch.tensor(np.concatenate([t.ravel() for t in truth]), dtype=torch.float32,
                                   device="cuda")
            out = torch.empty(len(r_ref), dtype=torch.float64, device="cuda")
            fit.residual_rms(truth_d, a, out)
            torch.cuda.synchronize()
            e_a = rel(a.double().cpu().numpy(), a_ref, f"alpha-sweep/commands/alpha{alpha}/frame{k}")
            e_r = rel(out.cpu().numpy(), r_ref, f"alpha-sweep/rms/alpha{alpha}/frame{k}")
            assert e_a < 1e-5, (alpha, k, e_a)
            assert e_r < 1e-5, (alpha, k, e_r)
            rms_g.append(float(out.mean()))
            rms_o.append(float(np.mean(r_ref)))
        gpu_curve[alpha] = float(np.mean(rms_g))
        ora_curve[alpha] = float(np.mean(rms_o))
        fit.close()
        plan.close()
    assert min(gpu_curve, key=gpu_curve.get) == min(ora_curve, key=ora_curve.get), (gpu_curve, ora_curve)
