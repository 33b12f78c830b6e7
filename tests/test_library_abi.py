"""The C-ABI library builds, loads and exports every symbol include/tomo.h
declares; host-side validation of geometries needs no GPU."""
import ctypes
import math
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tomo.h")


def _header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tomo_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1302_3734_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists(build.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    build.build()
    import paper_1302_3734_gb300 as pkg
    return pkg.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_1302_3734_gb300 import SIGNATURES
    assert sorted(n for n, _, _ in SIGNATURES) == _header_functions()


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.tomo_version()
    assert lib.tomo_last_error() is not None


def _status_of(geom):
    import paper_1302_3734_gb300 as pkg
    lib = pkg.load_library()
    g, keep = pkg.geometry_struct(geom)
    h = ctypes.c_void_p()
    st = lib.tomo_plan_create(ctypes.byref(g), None, ctypes.byref(h))
    if st == 0:
        lib.tomo_destroy(h)
    return st, lib.tomo_last_error().decode()


def test_validation_errors_without_gpu(lib):
    from synth import configs
    g = configs.small_lgs_config()
    g["levels"] = 5            # 32 / 2^4 = 2 < 6 taps
    st, msg = _status_of(g)
    assert st == 3 and "filter length" in msg
    g = configs.small_lgs_config()
    g["wfs"][0]["tt_only"] = True
    st, _ = _status_of(g)
    assert st == 1
    g = configs.small_lgs_config()
    g["layers"][0]["N"] = 48   # not a power of two
    st, _ = _status_of(g)
    assert st == 3
    g = configs.small_lgs_config()
    g["wfs"][1]["valid"][:] = 0
    st, msg = _status_of(g)
    assert st == 2 and "no valid subaperture" in msg
    g = configs.small_lgs_config(n_sub=16, N=16, dx=0.25)   # 8 m pupil on a 4 m grid
    st, msg = _status_of(g)
    assert st == 2 and "wider than the grid" in msg
    g = configs.small_lgs_config()
    g["layers"][2]["altitude"] = 95e3                        # above the sodium layer
    st, _ = _status_of(g)
    assert st == 2
    g = configs.small_lgs_config()
    g["wavelet_order"] = 7
    st, _ = _status_of(g)
    assert st == 1


def test_a_valid_geometry_reaches_the_device_step(lib):
    # without a GPU the only possible failure of a valid geometry is the CUDA step
    import torch
    from synth import configs
    st, msg = _status_of(configs.config1())
    if torch.cuda.is_available():
        assert st == 0, msg
    else:
        assert st == 5, msg


def test_server_argument_validation_without_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    for args in ((0, -1, 2, 8, 4), (0, 10, 0, 8, 4), (0, 10, 5, 8, 4), (0, 10, 2, 0, 4),
                 (0, 10, 2, 8, 0), (0, 10, 2, 300, 4)):
        assert lib.tomo_server_create(*args, ctypes.byref(h)) == 1, args
        assert not h.value
    assert lib.tomo_server_create(0, 10, 2, 8, 4, None) == 1
    # NULL servers are refused, not dereferenced
    assert lib.tomo_server_submit(None, 0, None, 0) == 1
    assert lib.tomo_server_release(None, 0) == 1
    assert lib.tomo_server_drain(None, 1.0) == 1
    assert lib.tomo_server_poll(None, None, 4) == 0
    lib.tomo_server_destroy(None)
    assert lib.tomo_server_clock() > 0.0


def test_plan_options_validation_without_gpu(lib):
    import ctypes
    from synth import configs
    from paper_1302_3734_gb300.binding import geometry_struct, PlanOptions
    g, keep = geometry_struct(configs.small_lgs_config())
    h = ctypes.c_void_p()
    opt = PlanOptions()
    opt.reserved[3] = 1
    assert lib.tomo_plan_create_ex(ctypes.byref(g), ctypes.byref(opt), None, ctypes.byref(h)) == 1
    opt = PlanOptions()
    for bad in (3, 32, 17):            # not a power of two, too large
        opt.cluster_size = bad
        assert lib.tomo_plan_create_ex(ctypes.byref(g), ctypes.byref(opt), None, ctypes.byref(h)) == 1
        assert "cluster size" in lib.tomo_last_error().decode()
    opt = PlanOptions()
    opt.transforms = 2                 # streamed: up to 64 gather bands, at most N/2
    for bad in (48, 128, 64):
        opt.cluster_size = bad
        assert lib.tomo_plan_create_ex(ctypes.byref(g), ctypes.byref(opt), None, ctypes.byref(h)) == 1
        assert "cluster size" in lib.tomo_last_error().decode()
    assert not h.value


def test_fit_and_control_argument_validation_without_gpu(lib):
    """The fitting, closed-loop and server-loop entry points refuse NULL objects and
    out-of-range arguments before touching a device."""
    import ctypes
    from synth import configs
    from paper_1302_3734_gb300.binding import fit_geometry_struct, geometry_struct, PlanOptions
    h = ctypes.c_void_p()
    g = configs.with_fitting(configs.small_lgs_config())
    fg, keep = fit_geometry_struct(g["fitting"])
    assert lib.tomo_fit_create(None, ctypes.byref(fg), ctypes.byref(h)) == 1
    assert not h.value
    assert lib.tomo_fit_apply_normal(None, None, None, None) == 1
    assert lib.tomo_fit_rhs(None, None, None, None) == 1
    assert lib.tomo_fit_residual_rms(None, None, None, None, None) == 1
    assert lib.tomo_fit_solve(None, None, None, 4, 0, None) == 1
    assert lib.tomo_reconstruct(None, None, None, None, 10, 4, 1, None) == 1
    assert lib.tomo_mirror_slopes(None, None, None, None, 1.0, None) == 1
    assert lib.tomo_polc_step(None, None, None, None, None, None, None, 0.4, 10, 4, 1, None) == 1
    assert lib.tomo_fit_get_info(None, None) == 1
    lib.tomo_fit_destroy(None)
    # the server refuses a closed-loop admission with a non-finite gain before building a plan
    gs, keep_g = geometry_struct(g)
    opt = PlanOptions()
    tid = ctypes.c_int(-1)
    assert lib.tomo_server_admit_loop(None, ctypes.byref(gs), ctypes.byref(opt), ctypes.byref(fg), 0.4, 4,
                                      ctypes.byref(tid)) == 1
    assert lib.tomo_server_get_fit(None, 0, ctypes.byref(h)) == 1
    assert "NULL" in lib.tomo_last_error().decode()
