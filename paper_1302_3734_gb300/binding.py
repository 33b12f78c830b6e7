"""ctypes binding of ``libtomo.so`` (include/tomo.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts a geometry ``dict`` (see ``synth.configs``) into the C structs, checks
tensor shapes/dtypes/devices, and passes raw device pointers and the current
CUDA stream.  There is no fallback: if the library is missing or a call fails,
an exception is raised.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtomo.so")

STATUS = {0: "TOMO_OK", 1: "TOMO_ERR_ARG", 2: "TOMO_ERR_GEOMETRY", 3: "TOMO_ERR_LEVELS",
          4: "TOMO_ERR_NOMEM", 5: "TOMO_ERR_CUDA", 6: "TOMO_ERR_TIMEOUT",
          7: "TOMO_ERR_BREAKDOWN", 8: "TOMO_ERR_UNSUPPORTED", 9: "TOMO_ERR_FULL",
          10: "TOMO_ERR_SUPERSEDED"}

KERNEL_KINDS = ("synthesis", "forward", "analysis", "update", "other", "gather")


class TomoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Wfs(ctypes.Structure):
    _fields_ = [("theta_x", ctypes.c_double), ("theta_y", ctypes.c_double),
                ("height", ctypes.c_double), ("n_sub", ctypes.c_int),
                ("d_sub", ctypes.c_double), ("valid", ctypes.POINTER(ctypes.c_ubyte)),
                ("sigma", ctypes.c_double), ("tt_only", ctypes.c_int),
                ("remove_tt", ctypes.c_int), ("elong_tau", ctypes.c_double),
                ("elong_scale", ctypes.c_double), ("llt_x", ctypes.c_double),
                ("llt_y", ctypes.c_double)]


class Layer(ctypes.Structure):
    _fields_ = [("altitude", ctypes.c_double), ("dx", ctypes.c_double),
                ("N", ctypes.c_int), ("prior_weight", ctypes.c_double)]


class Geometry(ctypes.Structure):
    _fields_ = [("D_tel", ctypes.c_double), ("obstruction", ctypes.c_double),
                ("n_wfs", ctypes.c_int), ("wfs", ctypes.POINTER(Wfs)),
                ("n_layers", ctypes.c_int), ("layers", ctypes.POINTER(Layer)),
                ("wavelet_order", ctypes.c_int), ("levels", ctypes.c_int),
                ("alpha", ctypes.c_double), ("L0", ctypes.c_double),
                ("precond", ctypes.c_int), ("precision", ctypes.c_int)]


class FrameResult(ctypes.Structure):
    _fields_ = [("telescope", ctypes.c_int), ("status", ctypes.c_int), ("tag", ctypes.c_longlong),
                ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch_size", ctypes.c_int),
                ("result_slot", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("frames_submitted", ctypes.c_longlong), ("frames_done", ctypes.c_longlong),
                ("frames_superseded", ctypes.c_longlong), ("launches", ctypes.c_longlong), ("bytes_in_use", ctypes.c_longlong),
                ("budget_bytes", ctypes.c_longlong), ("telescopes", ctypes.c_int),
                ("in_flight", ctypes.c_int)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int), ("transforms", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_coeffs", ctypes.c_longlong), ("n_slopes", ctypes.c_longlong),
                ("n_layers", ctypes.c_int), ("n_wfs", ctypes.c_int),
                ("cluster_size", ctypes.c_int), ("kernels_per_iteration", ctypes.c_int),
                ("kernels_per_solve_base", ctypes.c_int), ("device_bytes", ctypes.c_longlong),
                ("bytes_per_iteration", ctypes.c_longlong), ("precision", ctypes.c_int),
                ("breakdown_pending", ctypes.c_int), ("gather_separate", ctypes.c_int), ("streamed", ctypes.c_int)]


class Dm(ctypes.Structure):
    _fields_ = [("altitude", ctypes.c_double), ("pitch", ctypes.c_double), ("n", ctypes.c_int)]


class FitGeometry(ctypes.Structure):
    _fields_ = [("n_dm", ctypes.c_int), ("dms", ctypes.POINTER(Dm)), ("n_dir", ctypes.c_int),
                ("theta", ctypes.POINTER(ctypes.c_double)), ("n_sub", ctypes.c_int),
                ("d_sub", ctypes.c_double), ("valid", ctypes.POINTER(ctypes.c_ubyte))]


class FitInfo(ctypes.Structure):
    _fields_ = [("n_act", ctypes.c_longlong), ("n_active", ctypes.c_longlong),
                ("n_points", ctypes.c_int), ("n_dir", ctypes.c_int), ("n_dm", ctypes.c_int),
                ("kernels_per_iteration", ctypes.c_int), ("kernels_per_solve_base", ctypes.c_int),
                ("device_bytes", ctypes.c_longlong), ("normal_nonzeros", ctypes.c_longlong),
                ("bytes_per_iteration", ctypes.c_longlong)]


# (name, restype, argtypes) of every symbol declared in include/tomo.h
_VP = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = [
    ("tomo_plan_create", _I, [ctypes.POINTER(Geometry), _VP, ctypes.POINTER(_VP)]),
    ("tomo_plan_create_ex", _I, [ctypes.POINTER(Geometry), ctypes.POINTER(PlanOptions), _VP,
                                 ctypes.POINTER(_VP)]),
    ("tomo_solve", _I, [_VP, _VP, _VP, _I, _I, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("tomo_solve_batch", _I, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                              _I, _I, _I, _VP]),
    ("tomo_coeffs_to_layers", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_layers_to_coeffs", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_layers_to_slopes", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_apply_normal", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_rhs", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_jacobi_diagonal", _I, [_VP, _VP, _VP]),
    ("tomo_jacobi_diagonal_noalloc", _I, [_VP, ctypes.c_double, _VP, _VP]),
    ("tomo_plan_get_info", _I, [_VP, ctypes.POINTER(PlanInfo)]),
    ("tomo_plan_device_bytes", ctypes.c_size_t, [_VP]),
    ("tomo_set_kernel_timing", _I, [_VP, _I]),
    ("tomo_get_kernel_times", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), _I]),
    ("tomo_set_launch_mode", _I, [_VP, _I]),
    ("tomo_probe_l2_read", _I, [_VP, ctypes.c_longlong, _I, _I, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("tomo_launch_count", ctypes.c_longlong, []),
    ("tomo_last_error", ctypes.c_char_p, []),
    ("tomo_destroy", None, [_VP]),
    ("tomo_version", ctypes.c_char_p, []),
    ("tomo_server_create", _I, [ctypes.c_size_t, _I, _I, _I, _I, ctypes.POINTER(_VP)]),
    ("tomo_server_admit", _I, [_VP, ctypes.POINTER(Geometry), ctypes.POINTER(_I)]),
    ("tomo_server_admit_ex", _I, [_VP, ctypes.POINTER(Geometry), ctypes.POINTER(PlanOptions),
                                  ctypes.POINTER(_I)]),
    ("tomo_server_set_policy", _I, [_VP, _I]),
    ("tomo_server_release", _I, [_VP, _I]),
    ("tomo_server_submit", _I, [_VP, _I, _VP, ctypes.c_longlong]),
    ("tomo_server_poll", _I, [_VP, ctypes.POINTER(FrameResult), _I]),
    ("tomo_server_result", _I, [_VP, _I, _I, ctypes.c_longlong, _VP]),
    ("tomo_server_drain", _I, [_VP, ctypes.c_double]),
    ("tomo_server_get_stats", _I, [_VP, ctypes.POINTER(ServerStats)]),
    ("tomo_server_get_plan", _I, [_VP, _I, ctypes.POINTER(_VP)]),
    ("tomo_server_admit_loop", _I, [_VP, ctypes.POINTER(Geometry), ctypes.POINTER(PlanOptions),
                                    ctypes.POINTER(FitGeometry), ctypes.c_double, _I, ctypes.POINTER(_I)]),
    ("tomo_server_get_fit", _I, [_VP, _I, ctypes.POINTER(_VP)]),
    ("tomo_server_clock", ctypes.c_double, []),
    ("tomo_server_destroy", None, [_VP]),
    ("tomo_fit_create", _I, [_VP, ctypes.POINTER(FitGeometry), ctypes.POINTER(_VP)]),
    ("tomo_fit_get_info", _I, [_VP, ctypes.POINTER(FitInfo)]),
    ("tomo_fit_apply_normal", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_fit_rhs", _I, [_VP, _VP, _VP, _VP]),
    ("tomo_fit_residual_rms", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tomo_fit_solve", _I, [_VP, _VP, _VP, _I, _I, _VP]),
    ("tomo_reconstruct", _I, [_VP, _VP, _VP, _VP, _I, _I, _I, _VP]),
    ("tomo_mirror_slopes", _I, [_VP, _VP, _VP, _VP, ctypes.c_double, _VP]),
    ("tomo_polc_step", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, _I, _I, _I, _VP]),
    ("tomo_fit_destroy", None, [_VP]),
]

_lib = None


def load_library(path=LIB_PATH):
    """Load libtomo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1302_3734_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise TomoError(status, load_library().tomo_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def geometry_struct(geom):
    """C structs of a geometry dict; returns (Geometry, keep-alive list)."""
    keep = []
    ws = (Wfs * len(geom["wfs"]))()
    for i, w in enumerate(geom["wfs"]):
        ws[i].theta_x, ws[i].theta_y = float(w["theta"][0]), float(w["theta"][1])
        h = float(w["height"])
        ws[i].height = h if math.isfinite(h) else math.inf
        ws[i].n_sub = int(w["n_sub"])
        ws[i].d_sub = float(w["d_sub"])
        if w.get("valid") is not None:
            v = np.ascontiguousarray(np.asarray(w["valid"], dtype=np.uint8))
            if v.shape != (w["n_sub"], w["n_sub"]):
                raise ValueError("valid mask must be [n_sub, n_sub]")
            keep.append(v)
            ws[i].valid = v.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        else:
            ws[i].valid = None
        ws[i].sigma = float(w["sigma"])
        ws[i].tt_only = int(bool(w["tt_only"]))
        ws[i].remove_tt = int(bool(w["remove_tt"]))
        ws[i].elong_tau = float(w.get("elong_tau", 0.0))
        ws[i].elong_scale = float(w.get("elong_scale", 0.0))
        llt = w.get("llt", (0.0, 0.0))
        ws[i].llt_x, ws[i].llt_y = float(llt[0]), float(llt[1])
    ls = (Layer * len(geom["layers"]))()
    for i, lay in enumerate(geom["layers"]):
        ls[i].altitude = float(lay["altitude"])
        ls[i].dx = float(lay["dx"])
        ls[i].N = int(lay["N"])
        ls[i].prior_weight = float(lay["prior_weight"])
    keep += [ws, ls]
    g = Geometry(float(geom["D_tel"]), float(geom.get("obstruction", 0.0)), len(geom["wfs"]),
                 ws, len(geom["layers"]), ls, int(geom["wavelet_order"]), int(geom["levels"]),
                 float(geom["alpha"]), float(geom["L0"]), int(geom["precond"]),
                 int(geom["precision"]))
    return g, keep


class Plan:
    """One adaptive-optics system: tables, prior, Jacobi diagonal and workspace on the GPU."""

    def __init__(self, geom, stream=None, cluster_size=0, transforms=0):
        lib = load_library()
        g, keep = geometry_struct(geom)
        h = ctypes.c_void_p()
        opt = PlanOptions()
        opt.cluster_size = int(cluster_size)
        opt.transforms = int(transforms)
        _check(lib.tomo_plan_create_ex(ctypes.byref(g), ctypes.byref(opt), _stream(stream),
                                       ctypes.byref(h)))
        self._h = h
        self.info = self._info()
        self.n = int(self.info.n_coeffs)
        self.n_slopes = int(self.info.n_slopes)
        self.precision = int(self.info.precision)
        del keep

    @property
    def handle(self):
        return self._h

    def _info(self):
        inf = PlanInfo()
        _check(load_library().tomo_plan_get_info(self._h, ctypes.byref(inf)))
        return inf

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision else torch.float32

    def _tensor(self, t, n, name, dtype=None):
        dt = dtype or self.dtype
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}")
        if not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be contiguous with {n} elements")
        return ctypes.c_void_p(t.data_ptr())

    def solve(self, slopes, coeffs, iters, warm=True, stream=None, resnorm=False):
        """One frame; coeffs holds x0 (warm) and receives x.  Returns ||r|| when resnorm."""
        out = ctypes.c_double(0.0)
        _check(load_library().tomo_solve(
            self._h, self._tensor(slopes, self.n_slopes, "slopes"),
            self._tensor(coeffs, self.n, "coeffs"), int(iters), int(bool(warm)),
            _stream(stream), ctypes.byref(out) if resnorm else None))
        return out.value if resnorm else None

    def coeffs_to_layers(self, coeffs, layers, stream=None):
        _check(load_library().tomo_coeffs_to_layers(
            self._h, self._tensor(coeffs, self.n, "coeffs"), self._tensor(layers, self.n, "layers"),
            _stream(stream)))

    def layers_to_coeffs(self, layers, coeffs, stream=None):
        _check(load_library().tomo_layers_to_coeffs(
            self._h, self._tensor(layers, self.n, "layers"), self._tensor(coeffs, self.n, "coeffs"),
            _stream(stream)))

    def layers_to_slopes(self, layers, slopes, stream=None):
        _check(load_library().tomo_layers_to_slopes(
            self._h, self._tensor(layers, self.n, "layers"),
            self._tensor(slopes, self.n_slopes, "slopes"), _stream(stream)))

    def apply_normal(self, x, out, stream=None):
        _check(load_library().tomo_apply_normal(
            self._h, self._tensor(x, self.n, "x"), self._tensor(out, self.n, "out"), _stream(stream)))

    def rhs(self, slopes, out, stream=None):
        _check(load_library().tomo_rhs(
            self._h, self._tensor(slopes, self.n_slopes, "slopes"),
            self._tensor(out, self.n, "out"), _stream(stream)))

    def jacobi_diagonal(self, out, stream=None):
        import torch
        _check(load_library().tomo_jacobi_diagonal(
            self._h, self._tensor(out, self.n, "out", torch.float64), _stream(stream)))

    def jacobi_diagonal_noalloc(self, out, alpha, stream=None):
        """The Jacobi diagonal for `alpha`, computed without device allocation."""
        import torch
        _check(load_library().tomo_jacobi_diagonal_noalloc(
            self._h, float(alpha), self._tensor(out, self.n, "out", torch.float64), _stream(stream)))

    def device_bytes(self):
        return int(load_library().tomo_plan_device_bytes(self._h))

    def set_kernel_timing(self, enable):
        _check(load_library().tomo_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_times(self):
        """{kind: (launches, total ms)} since timing was (re)enabled."""
        k = len(KERNEL_KINDS)
        counts = (ctypes.c_int * k)()
        ms = (ctypes.c_double * k)()
        _check(load_library().tomo_get_kernel_times(self._h, counts, ms, k))
        return {name: (counts[i], ms[i]) for i, name in enumerate(KERNEL_KINDS)}

    def set_launch_mode(self, use_graphs):
        _check(load_library().tomo_set_launch_mode(self._h, int(bool(use_graphs))))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().tomo_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(plans, slopes, coeffs, iters, warm=True, stream=None):
    """Frames of several plans solved together (tomo_solve_batch)."""
    n = len(plans)
    ph = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    sp = (ctypes.c_void_p * n)(*[p._tensor(s, p.n_slopes, "slopes").value
                                 for p, s in zip(plans, slopes)])
    cp = (ctypes.c_void_p * n)(*[p._tensor(c, p.n, "coeffs").value for p, c in zip(plans, coeffs)])
    _check(load_library().tomo_solve_batch(ph, sp, cp, n, int(iters), int(bool(warm)), _stream(stream)))


def fit_geometry_struct(fit):
    """C structs of a fitting geometry dict (``geom["fitting"]``, see
    ``synth.configs.with_fitting``); returns (FitGeometry, keep-alive list)."""
    dms = (Dm * len(fit["dms"]))()
    for i, m in enumerate(fit["dms"]):
        dms[i].altitude, dms[i].pitch, dms[i].n = float(m["altitude"]), float(m["pitch"]), int(m["n"])
    th = np.ascontiguousarray(np.asarray(fit["directions"], dtype=np.float64).reshape(-1, 2))
    v = np.ascontiguousarray(np.asarray(fit["valid"], dtype=np.uint8))
    if v.shape != (fit["n_sub"], fit["n_sub"]):
        raise ValueError("valid mask must be [n_sub, n_sub]")
    g = FitGeometry(len(fit["dms"]), dms, th.shape[0], th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    int(fit["n_sub"]), float(fit["d_sub"]), v.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return g, [dms, th, v]


class Fit:
    """The fitting step of a plan (tomo_fit_*): mirror commands from the layers."""

    def __init__(self, plan, fit):
        lib = load_library()
        g, keep = fit_geometry_struct(fit)
        h = ctypes.c_void_p()
        _check(lib.tomo_fit_create(plan.handle, ctypes.byref(g), ctypes.byref(h)))
        del keep
        self._h = h
        self.plan = plan
        inf = FitInfo()
        _check(lib.tomo_fit_get_info(h, ctypes.byref(inf)))
        self.info = inf
        self.n = int(inf.n_act)

    def apply_normal(self, a, out, stream=None):
        p = self.plan
        _check(load_library().tomo_fit_apply_normal(
            self._h, p._tensor(a, self.n, "a"), p._tensor(out, self.n, "out"), _stream(stream)))

    def rhs(self, layers, out, stream=None):
        p = self.plan
        _check(load_library().tomo_fit_rhs(
            self._h, p._tensor(layers, p.n, "layers"), p._tensor(out, self.n, "out"), _stream(stream)))

    def residual_rms(self, layers, a, out, stream=None):
        """out (float64 CUDA tensor of n_dir): the piston-removed RMS of P_j phi - H_j a per
        direction (a = None: no correction)."""
        import torch
        p = self.plan
        _check(load_library().tomo_fit_residual_rms(
            self._h, p._tensor(layers, p.n, "layers"), None if a is None else p._tensor(a, self.n, "a"),
            p._tensor(out, int(self.info.n_dir), "out", torch.float64), _stream(stream)))

    def solve(self, layers, a, iters, warm=True, stream=None):
        """CG on H^T H a = H^T P phi; a holds the start (warm) and receives the commands."""
        p = self.plan
        _check(load_library().tomo_fit_solve(
            self._h, p._tensor(layers, p.n, "layers"), p._tensor(a, self.n, "a"), int(iters),
            int(bool(warm)), _stream(stream)))

    def reconstruct(self, slopes, coeffs, a, iters, fit_iters, warm=True, stream=None):
        """Slopes to mirror commands: the plan's solve, W^-1, then the fitting solve."""
        p = self.plan
        _check(load_library().tomo_reconstruct(
            self._h, p._tensor(slopes, p.n_slopes, "slopes"), p._tensor(coeffs, p.n, "coeffs"),
            p._tensor(a, self.n, "a"), int(iters), int(fit_iters), int(bool(warm)), _stream(stream)))

    def mirror_slopes(self, a, out, slopes_in=None, scale=1.0, stream=None):
        """out = slopes_in + scale * A_hat a (slopes_in None: 0)."""
        p = self.plan
        _check(load_library().tomo_mirror_slopes(
            self._h, p._tensor(a, self.n, "a"),
            None if slopes_in is None else p._tensor(slopes_in, p.n_slopes, "slopes_in"),
            p._tensor(out, p.n_slopes, "out"), float(scale), _stream(stream)))

    def polc_step(self, slopes, coeffs, a_rec, a_tm2, a_tm1, a_t, gain, iters, fit_iters, warm=True,
                  stream=None):
        """One step of pseudo-open-loop control (Algorithm 4.1) from the residual slopes."""
        p = self.plan
        _check(load_library().tomo_polc_step(
            self._h, p._tensor(slopes, p.n_slopes, "slopes"), p._tensor(coeffs, p.n, "coeffs"),
            p._tensor(a_rec, self.n, "a_rec"), p._tensor(a_tm2, self.n, "a_tm2"),
            p._tensor(a_tm1, self.n, "a_tm1"), p._tensor(a_t, self.n, "a_t"), float(gain), int(iters),
            int(fit_iters), int(bool(warm)), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().tomo_fit_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The served stream of tomo_server_*: telescopes admitted by device memory, frames
    submitted from host memory and solved warm-started, batched on arrival."""

    def __init__(self, budget_bytes=0, iters=10, max_in_flight=2, queue_depth=16, result_slots=8):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.tomo_server_create(int(budget_bytes), int(iters), int(max_in_flight),
                                      int(queue_depth), int(result_slots), ctypes.byref(h)))
        self._h = h
        self._info = {}
        self._n_out = {}
        self._buf = (FrameResult * 4096)()

    def admit(self, geom, cluster_size=0, transforms=0):
        """Admit a telescope; returns its id (TomoError with status TOMO_ERR_NOMEM when the
        budget does not allow it)."""
        lib = load_library()
        g, keep = geometry_struct(geom)
        tid = ctypes.c_int(-1)
        opt = PlanOptions()
        opt.cluster_size = int(cluster_size)
        opt.transforms = int(transforms)
        _check(lib.tomo_server_admit_ex(self._h, ctypes.byref(g), ctypes.byref(opt), ctypes.byref(tid)))
        del keep
        plan = ctypes.c_void_p()
        _check(lib.tomo_server_get_plan(self._h, tid.value, ctypes.byref(plan)))
        inf = PlanInfo()
        _check(lib.tomo_plan_get_info(plan, ctypes.byref(inf)))
        self._info[tid.value] = inf
        return tid.value

    def admit_loop(self, geom, gain=0.4, fit_iters=4, cluster_size=0):
        """Admit a telescope run in closed loop (pseudo-open-loop control with the mirrors of
        geom["fitting"]): its frames are residual slopes, its results mirror commands."""
        lib = load_library()
        g, keep = geometry_struct(geom)
        fg, keep_f = fit_geometry_struct(geom["fitting"])
        tid = ctypes.c_int(-1)
        opt = PlanOptions()
        opt.cluster_size = int(cluster_size)
        _check(lib.tomo_server_admit_loop(self._h, ctypes.byref(g), ctypes.byref(opt), ctypes.byref(fg),
                                          float(gain), int(fit_iters), ctypes.byref(tid)))
        del keep, keep_f
        plan = ctypes.c_void_p()
        _check(lib.tomo_server_get_plan(self._h, tid.value, ctypes.byref(plan)))
        inf = PlanInfo()
        _check(lib.tomo_plan_get_info(plan, ctypes.byref(inf)))
        fit = ctypes.c_void_p()
        _check(lib.tomo_server_get_fit(self._h, tid.value, ctypes.byref(fit)))
        fi = FitInfo()
        _check(lib.tomo_fit_get_info(fit, ctypes.byref(fi)))
        self._info[tid.value] = inf
        self._n_out[tid.value] = int(fi.n_act)
        return tid.value

    def info(self, telescope):
        return self._info[telescope]

    def set_policy(self, latest_only):
        """True: solve only the newest waiting frame of a telescope; older ones come back with
        status TOMO_ERR_SUPERSEDED."""
        _check(load_library().tomo_server_set_policy(self._h, int(bool(latest_only))))

    def release(self, telescope):
        _check(load_library().tomo_server_release(self._h, int(telescope)))
        self._info.pop(telescope, None)
        self._n_out.pop(telescope, None)

    def submit(self, telescope, slopes, tag):
        """slopes: C-contiguous host array (float32, or float64 for precision-1 plans) of
        n_slopes elements.  Returns False when the telescope's queue is full."""
        inf = self._info[telescope]
        dt = np.float64 if inf.precision else np.float32
        if slopes.dtype != dt or not slopes.flags.c_contiguous or slopes.size != inf.n_slopes:
            raise ValueError(f"slopes must be a contiguous {np.dtype(dt).name} array of {inf.n_slopes}")
        st = load_library().tomo_server_submit(self._h, int(telescope),
                                                ctypes.c_void_p(slopes.ctypes.data), int(tag))
        if st == 9:
            return False
        _check(st)
        return True

    def poll(self):
        """Finished frames: a list of dicts (telescope, status, tag, t_submit, t_launch,
        t_done, batch_size, result_slot)."""
        out = []
        lib = load_library()
        while True:
            k = lib.tomo_server_poll(self._h, self._buf, len(self._buf))
            for i in range(k):
                r = self._buf[i]
                out.append({f: getattr(r, f) for f, _ in FrameResult._fields_})
            if k < len(self._buf):
                return out

    def result(self, telescope, result_slot, tag):
        """The result of a finished frame (numpy array): coefficients, or the mirror commands of
        a closed-loop telescope; None if the slot moved on."""
        inf = self._info[telescope]
        n = self._n_out.get(telescope, int(inf.n_coeffs))
        out = np.empty(n, dtype=np.float64 if inf.precision else np.float32)
        st = load_library().tomo_server_result(self._h, int(telescope), int(result_slot), int(tag),
                                                ctypes.c_void_p(out.ctypes.data))
        return out if st == 0 else None

    def drain(self, timeout_s=60.0):
        _check(load_library().tomo_server_drain(self._h, float(timeout_s)))

    def stats(self):
        st = ServerStats()
        _check(load_library().tomo_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    @staticmethod
    def clock():
        return float(load_library().tomo_server_clock())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().tomo_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count():
    return int(load_library().tomo_launch_count())


def probe_l2_read(buf, passes=8, reps=20, stream=None):
    """L2 read bandwidth (GB/s) measured on the CUDA tensor `buf` (it should fit the L2)."""
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    out = ctypes.c_double(0.0)
    _check(load_library().tomo_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                             int(passes), int(reps), _stream(stream), ctypes.byref(out)))
    return out.value


def version():
    return load_library().tomo_version().decode()
