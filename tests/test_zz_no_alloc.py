"""The allocation-free Jacobi diagonal (tomo_jacobi_diagonal_noalloc) against
the diagonal the plan computed at creation (tomo_jacobi_diagonal), through the
C ABI, on two calls in a row.

Callers that cannot allocate device memory when they need the diagonal again
(a real-time thread retuning the regularisation weight, code inside another
framework's memory pool) use this entry point; its scratch is a fixed device
array of the library, so consecutive calls reuse the same memory and must give
the same result.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["eelt", "small"])
def test_noalloc_diagonal_matches_the_plan(which):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    geom = configs.config1() if which == "eelt" else configs.small_lgs_config()
    plan = pkg.Plan(geom)
    lib = pkg.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = torch.empty(plan.n, dtype=torch.float64, device="cuda")
    assert lib.tomo_jacobi_diagonal(plan.handle, ctypes.c_void_p(ref.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((plan.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.tomo_jacobi_diagonal_noalloc(plan.handle, ctypes.c_double(geom["alpha"]),
                                              ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.tomo_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref_h) / np.linalg.norm(ref_h)
        assert err < 1e-12, (call, err)
    plan.close()
