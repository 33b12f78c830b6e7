"""The allocation-free Jacobi diagonal (tomo_jacobi_diagonal_noalloc), called
through the C ABI.

Who needs it: a caller that cannot allocate device memory at the moment it
needs the diagonal again.  A real-time control thread that retunes the
regularisation weight alpha between frames must not take the latency of
cudaMalloc (which can serialise with the whole device), and code running inside
another framework's memory pool may have no allocator of its own.  The entry
point keeps its scratch in a fixed device array of the library, so consecutive
calls reuse the same memory and must give the same result.

Checked here, each on two calls in a row:
- at the plan's own alpha, against the diagonal the plan computed at creation
  (tomo_jacobi_diagonal);
- at other alphas (0, alpha/2, 2 alpha), against the FP64 oracle's diagonal
  built for that alpha, and on a tiny grid against the brute-force definition
  (one unit vector per coefficient);
- on the E-ELT plan, J(alpha') - J(alpha) = (alpha' - alpha) D with the
  oracle's prior D;
- a negative, NaN or infinite alpha is refused with TOMO_ERR_ARG, and a plan
  whose scratch exceeds the fixed array (the 100 m system with 60 layers) with
  TOMO_ERR_UNSUPPORTED, leaving the output untouched.

This file is collected last on purpose: pytest -x has run every other test
before it.
"""
import ctypes

import numpy as np
import pytest

from oracle import Tomography
from synth import configs

pytestmark = pytest.mark.gpu

TOMO_ERR_ARG = 1
TOMO_ERR_UNSUPPORTED = 8


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg, pkg.load_library()


def _noalloc(torch, lib, plan, alpha):
    """Two calls in a row at `alpha`; both results as numpy arrays."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for _ in range(2):
        out = torch.full((plan.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.tomo_jacobi_diagonal_noalloc(plan.handle, ctypes.c_double(alpha),
                                              ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.tomo_last_error().decode()
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    return outs


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("which", ["eelt", "small"])
def test_noalloc_diagonal_matches_the_plan(lib, which):
    torch, pkg, L = lib
    geom = configs.config1() if which == "eelt" else configs.small_lgs_config()
    plan = pkg.Plan(geom)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = torch.empty(plan.n, dtype=torch.float64, device="cuda")
    assert L.tomo_jacobi_diagonal(plan.handle, ctypes.c_void_p(ref.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    for call, got in enumerate(_noalloc(torch, L, plan, geom["alpha"])):
        err = _rel(got, ref_h)
        assert err < 1e-12, (call, err)
    plan.close()


@pytest.mark.parametrize("factor", [0.0, 0.5, 2.0])
def test_noalloc_diagonal_at_a_new_alpha_matches_the_oracle(lib, factor):
    torch, pkg, L = lib
    geom = configs.small_lgs_config()
    alpha = factor * geom["alpha"]
    ref = Tomography(dict(geom, alpha=alpha)).jacobi_diagonal()
    plan = pkg.Plan(geom)
    for call, got in enumerate(_noalloc(torch, L, plan, alpha)):
        err = _rel(got, ref)
        assert err < 1e-12, (factor, call, err)
    plan.close()


def test_noalloc_diagonal_at_a_new_alpha_matches_the_definition(lib):
    """Tiny grid: the oracle's brute-force diagonal (one unit vector per
    coefficient through Gamma P W^-1) at alpha' = 3 alpha."""
    torch, pkg, L = lib
    geom = configs.small_lgs_config(n_sub=8, N=16, n_layers=2, levels=2)
    alpha = 3.0 * geom["alpha"]
    ref = Tomography(dict(geom, alpha=alpha)).jacobi_diagonal_probe()
    plan = pkg.Plan(geom)
    for call, got in enumerate(_noalloc(torch, L, plan, alpha)):
        err = _rel(got, ref)
        assert err < 1e-12, (call, err)
    plan.close()


def test_noalloc_eelt_diagonal_moves_by_the_prior(lib):
    """E-ELT plan: the diagonal at 2 alpha minus the plan's diagonal is alpha D."""
    torch, pkg, L = lib
    geom = configs.config1()
    plan = pkg.Plan(geom)
    base = _noalloc(torch, L, plan, geom["alpha"])[0]
    D = Tomography(geom).prior_diagonal()
    for call, got in enumerate(_noalloc(torch, L, plan, 2.0 * geom["alpha"])):
        err = _rel(got - base, geom["alpha"] * D)
        assert err < 1e-12, (call, err)
    plan.close()


def test_noalloc_refuses_bad_alpha_and_oversized_plans(lib):
    torch, pkg, L = lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    plan = pkg.Plan(configs.small_lgs_config())
    out = torch.full((plan.n,), 7.0, dtype=torch.float64, device="cuda")
    for bad in (-1.0, float("nan"), float("inf")):
        st = L.tomo_jacobi_diagonal_noalloc(plan.handle, ctypes.c_double(bad),
                                            ctypes.c_void_p(out.data_ptr()), stream)
        assert st == TOMO_ERR_ARG, (bad, st)
    plan.close()
    # the 100 m system with 60 layers (25 of its layers repeated): 4.8 MB of basis
    # profiles and corner fractions, above the 4 MiB array
    g4 = configs.config4()
    big = pkg.Plan(dict(g4, layers=g4["layers"] + g4["layers"][1:26]))
    out = torch.full((big.n,), 7.0, dtype=torch.float64, device="cuda")
    st = L.tomo_jacobi_diagonal_noalloc(big.handle, ctypes.c_double(1.0),
                                        ctypes.c_void_p(out.data_ptr()), stream)
    assert st == TOMO_ERR_UNSUPPORTED, st
    msg = L.tomo_last_error().decode()
    assert "maximum" in msg and "bytes" in msg, msg
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    big.close()
