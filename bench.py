"""Benchmark: wavelet-domain MAP tomography frames on GB300 (one JSON line).

Workload (default): the E-ELT-sized MCAO system - 42 m pupil with 28 % of the
area obstructed, six sodium LGS (84x84 Shack-Hartmann, 90 km, cone effect,
tip/tilt removed) on a 1'-radius hexagon, three tip/tilt-only NGS at 1', nine
layers of 128^2 at 0.5 m, db3 with 4 levels, modified-Jacobi PCG with 10
iterations warm-started from the previous frame (Sec. 5.1 of the paper).
Frames come from seeded von Karman screens advected by frozen flow at 500 Hz;
slopes are the library's own noise-free measurement plus seeded noise.

A step is one frame (right-hand side, initial residual, 10 PCG iterations).
``value`` is frames solved per second with inputs resident in HBM; L2 is
flushed (a 256 MiB write) before every timed step, outside the timed window.

Further legs of the same line: ``batched`` (16 E-ELT systems, and 64 systems of
uneven size, per launch), ``large`` (the 100 m system), ``closed_loop`` (the
E-ELT system with its three mirrors: fitting and pseudo-open-loop control per
frame, with the Strehl ratio of the correction), ``served`` (16 telescopes
streaming frames through the server) and ``served_closed_loop`` (4 E-ELT
telescopes in closed loop through the server, each with a plant on the GPU).

``--impl reference`` times the FP64 CPU oracle on the same frames instead.
Under torchrun every rank solves its own independent telescope stream (weak
scaling, no data-path collective).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tomography solves/s and p99 frame latency at 84x84 MCAO vs plain GPU PCG"


# DRAM bytes (read + write) per launch of each PCG kernel on this workload, from one ncu capture
# with flushed caches, valid only for the kernel sources they were taken from (a SHA-256 over
# these files of paper_1302_3734_gb300/csrc, in this order).
NCU_TRAFFIC = {
    "sources": ["kernels.cu", "transform.cuh", "device_util.cuh", "adjoint.cuh", "common.h"],
    "sha256": "e8bcd2fe627f0f1f28c3a5b33cdb90d1ccbe9aea8a6d05076a506424cac1c457",
    "bytes": {"analysis": 5139456, "synthesis": 1843456, "forward": 749312, "update": 2985728},
}


def sources_digest():
    import hashlib
    h = hashlib.sha256()
    for name in NCU_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_1302_3734_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(kind):
    try:
        digest = sources_digest()
    except OSError:
        return None
    return NCU_TRAFFIC["bytes"].get(kind) if digest == NCU_TRAFFIC["sha256"] else None


def l2_probe(pkg, torch, dev):
    """L2 read bandwidth: the library's probe reads a 64 MiB buffer (resident in the 129 MB L2)
    16 times per launch over 20 launches, loads bypassing L1, timed with CUDA events; best of 3.
    (On GB300: 14 TB/s with 24 MiB and 8 passes, where launch overheads still count; 18.8 TB/s
    with 96 MiB; 7.0 TB/s with 512 MiB, which no longer fits and reads HBM.)"""
    a = torch.ones(16 << 20, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    return max(pkg.probe_l2_read(a, passes=16, reps=20, stream=stream) for _ in range(3))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch", type=int, default=16, help="E-ELT instances per batched solve")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 100 m configuration")
    ap.add_argument("--no-loop", action="store_true", help="skip the E-ELT closed loop with fitting")
    ap.add_argument("--loop-frames", type=int, default=120)
    ap.add_argument("--profile-leg", default=None, choices=["eelt", "batch16", "uneven64", "large"],
                    help="run only this workload's solves (no JSON line), for kernel profiles")
    ap.add_argument("--solves", type=int, default=3, help="solves of --profile-leg")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the served 16-telescope stream (0: skip it)")
    return ap.parse_args()


def workload():
    from synth import configs
    g = configs.config1()
    return g, {"workload": "E-ELT MCAO 42m, 6 LGS 84x84 @90km + 3 TT NGS, 9 layers 128^2 @0.5m, "
                           "db3 J=4, Jacobi PCG 10 it, warm start, 500 Hz frozen flow",
               "n_coeffs": sum(l["N"] ** 2 for l in g["layers"]), "iters": g["iters"],
               "precision": "FP32 operator and vectors; in-block dot products as float-float pairs "
                            "(about 48 bits); FP64 cross-block partials, alpha, beta and norms"}


def frame_screens(geom, k, rank):
    from synth import FrozenFlow
    if not hasattr(frame_screens, "ff"):
        frame_screens.ff = FrozenFlow(geom, 1, instance=rank)
    return frame_screens.ff.layers(k * 0.002)


def max_over_ranks(value_ms, dist, device):
    """The slowest rank's time: the job ends when its last rank does."""
    if not dist:
        return value_ms
    import torch
    t = torch.tensor([value_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, steps, tot_ms):
    """Whole-job solves per second: every rank solves `steps` frames in the slowest rank's time."""
    return ws * steps / (tot_ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _oracle_chain(args):
    """One process: the FP64 oracle solving a warm-started chain of frames for budget_s."""
    geom, frames_s, budget_s = args
    from oracle import Tomography
    ora = Tomography(geom)
    jd = ora.jacobi_diagonal()
    x = np.zeros(ora.n)
    n = 0
    t0 = time.perf_counter()
    while True:
        x = ora.pcg(ora.rhs(frames_s[n % len(frames_s)]), x, int(geom["iters"]), jd)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return n, time.perf_counter() - t0


def cpu_baseline(geom, frames_s, x0, budget_s):
    """The FP64 oracle solving the same frames on the host: one core, then one independent
    frame chain per host core (spawned processes), and the other configurations' single-core
    rates on bounded samples."""
    import multiprocessing as mp
    from oracle import Tomography
    from synth import configs, gaussian_noise
    t0 = time.perf_counter()
    ora = Tomography(geom)
    Jd = ora.jacobi_diagonal()
    plan_s = time.perf_counter() - t0
    x = np.asarray(x0, dtype=np.float64)
    n = 0
    t0 = time.perf_counter()
    while True:
        x = ora.pcg(ora.rhs(frames_s[n % len(frames_s)]), x, int(geom["iters"]), Jd)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": n / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} consecutive frames of the same workload, 10 FP64 PCG iterations each, "
                     f"numpy single core; plan (exact Jacobi diagonal) {plan_s:.2f}s excluded",
           "nproc": os.cpu_count()}
    # every host core: independent warm-started chains, one per process
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_chain, [(geom, frames_s, budget_s)] * cores)
    out["all_cores"] = {"value": sum(k / t for k, t in res), "unit": "solves/s", "cores": cores,
                        "sample": f"{cores} processes, each a chain of the same frames for "
                                  f"{budget_s:.0f} s ({sum(k for k, _ in res)} solves)"}
    # the 8 m configuration (30 CG iterations) and one PCG iteration of the 100 m one
    other = {}
    g0 = configs.config0()
    o0 = Tomography(g0)
    s0 = gaussian_noise(int(o0.meas_offsets[-1]), 0.1, 11)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < min(5.0, budget_s):
        o0.pcg(o0.rhs(s0), np.zeros(o0.n), int(g0["iters"]))
        k += 1
    other["cfg0_solves_per_s"] = k / (time.perf_counter() - t0)
    g4 = configs.config4()
    o4 = Tomography(g4)
    s4 = gaussian_noise(int(o4.meas_offsets[-1]), 0.3, 12)
    t0 = time.perf_counter()
    b4 = o4.rhs(s4)
    t_rhs = time.perf_counter() - t0
    t0 = time.perf_counter()
    o4.apply_normal(b4)
    t_op = time.perf_counter() - t0
    it4 = int(g4["iters"])
    other["cfg4_solves_per_s_estimated"] = 1.0 / (t_rhs + it4 * t_op)
    other["cfg4_sample"] = (f"right-hand side {t_rhs:.1f} s and one normal-operator apply {t_op:.1f} s "
                            f"timed; a {it4}-iteration cold solve is taken as the right-hand side plus "
                            f"{it4} applies (the vector updates are negligible beside them)")
    out["other_configs"] = other
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import Tomography
    from synth import gaussian_noise
    geom, cfg = workload()
    ora = Tomography(geom)
    Jd = ora.jacobi_diagonal()
    frames = []
    for k in range(args.warmup + args.steps):
        s = ora.measure(frame_screens(geom, k, 0)) + gaussian_noise(
            ora.meas_offsets[-1], 0.3, 1_000_000 + k)
        frames.append(s)
    x = np.zeros(ora.n)
    for k in range(args.warmup):
        x = ora.pcg(ora.rhs(frames[k]), x, int(geom["iters"]), Jd)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        x = ora.pcg(ora.rhs(frames[args.warmup + k]), x, int(geom["iters"]), Jd)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "latency_ms": {"p50": 1000 * float(np.percentile(times, 50)),
                           "p99": 1000 * float(np.percentile(times, 99))},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} frames, FP64 numpy oracle, single core"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def launch_bytes(plans, geoms):
    """Algorithmic bytes of one launch of each PCG kernel kind over the given plans (inputs read,
    outputs written, each once): synthesis reads r, J^-1, p and writes p, phi (5n); the forward
    kernel reads phi and writes the corner fields (n + V); the fused gather + analysis reads v, p
    and writes q (2n + V); where the gather runs separately it reads v and writes the gathered
    grids (n + V) and the analysis reads those and p and writes q (3n); the update reads x, r, p,
    q, J^-1 and writes x, r (7n).  V: corner values of the sensors that are not tip/tilt-only."""
    out = {"synthesis": 0, "forward": 0, "analysis": 0, "update": 0, "gather": 0}
    for p, g in zip(plans, geoms):
        e = 8 if p.precision else 4
        n = p.n
        V = (p.info.bytes_per_iteration // e - (15 if g["precond"] else 13) * n) // 2
        split = bool(p.info.gather_separate)
        out["synthesis"] += 5 * n * e
        out["forward"] += (n + V) * e
        out["analysis"] += (3 * n if split else 2 * n + V) * e
        out["gather"] += (n + V) * e if split else 0
        out["update"] += 7 * n * e
    return out


def kernel_roofline(kt, per_launch, peak, note=None):
    """The dominant kernel (by event time) of per-kind CUDA-event timings kt {kind: (launches, ms)}:
    its algorithmic bytes per launch over its mean launch time, against the HBM peak."""
    kinds = [k for k in per_launch if kt.get(k, (0, 0.0))[0] > 0 and per_launch[k] > 0]
    dom = max(kinds, key=lambda k: kt[k][1])
    cnt, ms = kt[dom]
    achieved = per_launch[dom] * cnt / (ms / 1000.0) / 1e9
    out = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "bytes_per_launch": per_launch[dom],
           "kernel_us_per_launch": {k: 1000.0 * kt[k][1] / kt[k][0] for k in kinds},
           "share_of_kernel_time": {k: kt[k][1] / sum(kt[j][1] for j in kinds) for k in kinds}}
    if note:
        out["note"] = note
    return out


def _timed_kinds(pkg, torch, plans, run, flush, reps):
    """Per-kind CUDA-event kernel times of `reps` calls of run(), timing on the first plan."""
    plans[0].set_kernel_timing(True)
    for k in range(reps):
        flush.fill_(float(k))
        run()
    kt = plans[0].kernel_times()
    plans[0].set_kernel_timing(False)
    return kt


def _time_batch(pkg, torch, plans, slopes, xs, iters, flush, steps, warmup):
    for _ in range(warmup):
        pkg.solve_batch(plans, slopes, xs, iters, warm=True)
    torch.cuda.synchronize()
    times = []
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.solve_batch(plans, slopes, xs, iters, warm=True)
        e1.record()
        times.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def bench_batched(pkg, torch, geom, slopes, flush, iters, args, peak, dev):
    """Many instances per launch: B E-ELT systems, and the 64 uneven instances."""
    from synth import configs, gaussian_noise
    out = {}
    steps = max(5, min(args.steps, 100))
    from paper_1302_3734_gb300.autotune import tune, _plans
    # B E-ELT instances, each on its own frame of the stream, at the tuned cluster size
    B = args.batch
    (c_e, tf_e), tab_e = tune([geom] * B, iters)
    plans = _plans([geom] * B, c_e, tf_e)
    F = slopes.shape[0]
    sl = [slopes[(3 * i) % F].clone() for i in range(B)]
    xs = [torch.zeros(plans[0].n, dtype=torch.float32, device=dev) for _ in range(B)]
    t = _time_batch(pkg, torch, plans, sl, xs, iters, flush, steps, 3)
    ms = float(np.mean(t))
    bytes_it = sum(p.info.bytes_per_iteration for p in plans)
    kt = _timed_kinds(pkg, torch, plans, lambda: pkg.solve_batch(plans, sl, xs, iters, warm=True), flush, 3)
    out["eelt"] = {"instances": B, "solves_per_s": B * 1000.0 / ms, "ms_per_batch": ms,
                   "cluster_size": c_e, "transforms": "streamed" if tf_e == 2 else "cluster",
                   "autotune_solves_per_s": tab_e,
                   "autotune_note": "keys: cluster size / transforms (1 cluster kernels, 2 streamed passes)",
                   "p99_ms": float(np.percentile(t, 99)),
                   "achieved_GBps_per_iteration_bytes": bytes_it * iters / (ms / 1000.0) / 1e9,
                   "frac_of_hbm_peak": bytes_it * iters / (ms / 1000.0) / 1e9 / peak,
                   "roofline": kernel_roofline(kt, launch_bytes(plans, [geom] * B), peak,
                                               "events around every launch of 3 batched solves (direct "
                                               "launches), L2 flushed before each")}
    for p in plans:
        p.close()
    # the 64-instance uneven workload
    geoms = configs.config2()
    (c_u, tf_u), tab_u = tune(geoms, 10)
    plans = _plans(geoms, c_u, tf_u)
    sl = []
    for i, (g, p) in enumerate(zip(geoms, plans)):
        sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                              for w in g["wfs"]])
        sl.append(torch.tensor(gaussian_noise(p.n_slopes, 1.0, 3_000_000 + i) * sig,
                               dtype=torch.float32, device=dev))
    xs = [torch.zeros(p.n, dtype=torch.float32, device=dev) for p in plans]
    t = _time_batch(pkg, torch, plans, sl, xs, 10, flush, steps, 3)
    ms = float(np.mean(t))
    bytes_it = sum(p.info.bytes_per_iteration for p in plans)
    kt = _timed_kinds(pkg, torch, plans, lambda: pkg.solve_batch(plans, sl, xs, 10, warm=True), flush, 3)
    out["uneven64"] = {"instances": len(plans), "solves_per_s": len(plans) * 1000.0 / ms,
                       "roofline": kernel_roofline(kt, launch_bytes(plans, geoms), peak,
                                                   "events around every launch of 3 batched solves "
                                                   "(direct launches), L2 flushed before each"),
                       "cluster_size": c_u, "transforms": "streamed" if tf_u == 2 else "cluster",
                       "autotune_solves_per_s": tab_u,
                       "ms_per_batch": ms, "p99_ms": float(np.percentile(t, 99)),
                       "coefficients": int(sum(p.n for p in plans)),
                       "achieved_GBps_per_iteration_bytes": bytes_it * 10 / (ms / 1000.0) / 1e9,
                       "frac_of_hbm_peak": bytes_it * 10 / (ms / 1000.0) / 1e9 / peak}
    for p in plans:
        p.close()
    return out


def bench_large(pkg, torch, dev, flush, peak, steps=5, warmup=2):
    """The 100 m stress configuration (35 layers of 512^2, db4 J=5, 20 PCG iterations):
    one instance, and a batch of four."""
    from synth import configs, gaussian_noise
    g = configs.config4()
    iters = int(g["iters"])
    out = {"workload": "100 m, 9 LGS 200x200 + 3 TT NGS, 35 layers 512^2, db4 J=5, Jacobi PCG "
                       f"{iters} it, cold start", "n_coeffs": sum(l["N"] ** 2 for l in g["layers"])}
    plans = [pkg.Plan(g) for _ in range(4)]
    sl = [torch.tensor(gaussian_noise(plans[0].n_slopes, 0.3, 6_000_000 + i), dtype=torch.float32,
                       device=dev) for i in range(4)]
    xs = [torch.zeros(plans[0].n, dtype=torch.float32, device=dev) for _ in range(4)]
    bytes_it = plans[0].info.bytes_per_iteration
    for label, k in (("single", 1), ("batch4", 4)):
        def once():
            if k == 1:
                plans[0].solve(sl[0], xs[0], iters, warm=False)
            else:
                pkg.solve_batch(plans, sl, xs, iters, warm=False)
        for _ in range(warmup):
            once()
        torch.cuda.synchronize()
        t = []
        for j in range(steps):
            flush.fill_(float(j))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            once()
            e1.record()
            t.append((e0, e1))
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in t]))
        gbs = k * bytes_it * iters / (ms / 1000.0) / 1e9
        kt = _timed_kinds(pkg, torch, plans, once, flush, 2)
        out[label] = {"solves_per_s": k * 1000.0 / ms, "ms": ms, "achieved_GBps_per_iteration_bytes": gbs,
                      "frac_of_hbm_peak": gbs / peak,
                      "roofline": kernel_roofline(kt, launch_bytes(plans[:k], [g] * k), peak,
                                                  "events around every launch of 2 solves (direct launches), "
                                                  "L2 flushed before each")}
    for p in plans:
        p.close()
    return out


def bench_closed_loop(pkg, torch, dev, flush, frames, gain=0.4, fit_iters=4):
    """The reconstruction and pseudo-open-loop control of Secs. 4.1-4.2 on the E-ELT system with
    its three mirrors (0, 4 and 12.7 km, 9296 actuators reached) and the 5 x 5 directions of a 2'
    field: each frame the sensors measure the frozen-flow atmosphere minus the mirror shapes
    applied two frames earlier, and one tomo_polc_step (mirror slopes, 10 warm PCG iterations,
    W^-1, 4 warm fitting CG iterations, control update; one CUDA graph) computes the next
    commands.  Timed: the control step (CUDA events, L2 flushed before each).  Quality: the
    Marechal Strehl at 2200 nm of the residual wavefront in the 25 directions, from
    tomo_fit_residual_rms, averaged over the second half of the frames (long exposure), with
    and without the correction."""
    from synth import configs, FrozenFlow, gaussian_noise
    g = configs.with_fitting(configs.config1())
    plan = pkg.Plan(g)
    fit = pkg.Fit(plan, g["fitting"])
    n, ns, na = plan.n, plan.n_slopes, fit.n
    nd = int(fit.info.n_dir)
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in g["wfs"]])
    flow = FrozenFlow(g, 1, instance=7)
    truth = torch.empty((frames, n), dtype=torch.float32, device=dev)
    meas = torch.empty((frames, ns), dtype=torch.float32, device=dev)
    for t in range(frames):
        truth[t].copy_(torch.from_numpy(np.concatenate([p.ravel() for p in flow.layers(0.002 * t)])
                                        .astype(np.float32)))
        plan.layers_to_slopes(truth[t], meas[t])
        meas[t] += torch.from_numpy((gaussian_noise(ns, 1.0, 5_000_000 + t) * sig).astype(np.float32)).to(dev)
    buf = [torch.zeros(na, dtype=torch.float32, device=dev) for _ in range(2)]
    x = torch.zeros(n, dtype=torch.float32, device=dev)
    rec = torch.zeros(na, dtype=torch.float32, device=dev)
    s = torch.empty(ns, dtype=torch.float32, device=dev)
    rms = torch.empty((frames, nd), dtype=torch.float64, device=dev)
    rms_open = torch.empty((frames, nd), dtype=torch.float64, device=dev)
    times = []
    for t in range(frames):
        a_tm2, a_tm1 = buf[t % 2], buf[(t + 1) % 2]
        fit.mirror_slopes(a_tm2, s, slopes_in=meas[t], scale=-1.0)
        fit.residual_rms(truth[t], a_tm2, rms[t])
        fit.residual_rms(truth[t], None, rms_open[t])
        flush.fill_(float(t))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fit.polc_step(s, x, rec, a_tm2, a_tm1, a_tm2, gain, 10, fit_iters, warm=t > 0)
        e1.record()
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in times])
    le = slice(frames // 2, frames)
    strehl = np.exp(-(rms.cpu().numpy()[le] * (500.0 / 2200.0)) ** 2).mean(axis=0)
    strehl_open = np.exp(-(rms_open.cpu().numpy()[le] * (500.0 / 2200.0)) ** 2).mean(axis=0)
    # the fitting step alone, on the last reconstructed layers
    lay = torch.empty(n, dtype=torch.float32, device=dev)
    plan.coeffs_to_layers(x, lay)
    a = torch.zeros(na, dtype=torch.float32, device=dev)
    ft = []
    for k in range(60):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fit.solve(lay, a, fit_iters, warm=True)
        e1.record()
        ft.append((e0, e1))
    torch.cuda.synchronize()
    fit_ms = np.array([a0.elapsed_time(b0) for a0, b0 in ft[10:]])
    # the fitting CG's iterations against the bytes they must move (H^T H and the vectors; the
    # right-hand side's two launches are left out of the bytes and counted in the time)
    fit_gbs = int(fit.info.bytes_per_iteration) * fit_iters / (float(fit_ms.mean()) / 1000.0) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    l2 = l2_probe(pkg, torch, dev)
    out = {"frames": frames, "gain": gain, "fit_iters": fit_iters, "tomo_iters": 10,
           "actuators": na, "actuators_reached": int(fit.info.n_active), "directions": nd,
           "control_steps_per_s": 1000.0 / float(ms[5:].mean()),
           "control_step_ms": {"p50": float(np.percentile(ms[5:], 50)), "p99": float(np.percentile(ms[5:], 99))},
           "fitting_ms": {"mean": float(fit_ms.mean()), "p99": float(np.percentile(fit_ms, 99))},
           "fitting_roofline": {"bytes_per_iteration": int(fit.info.bytes_per_iteration),
                                "normal_nonzeros": int(fit.info.normal_nonzeros),
                                "achieved_GBps": fit_gbs, "frac_of_hbm_peak": fit_gbs / hbm,
                                "frac_of_l2_peak": fit_gbs / l2,
                                "note": "L2-resident (H^T H is 10.8 MB); latency-bound at 10 launches per solve"},
           "strehl_2200nm_long_exposure": {"field_average": float(strehl.mean()),
                                           "on_axis": float(strehl[nd // 2]),
                                           "uncorrected_field_average": float(strehl_open.mean())},
           "note": "synthetic frozen-flow atmosphere (von Karman, r0 0.15 m, L0 25 m), not OCTOPUS: "
                   "the Strehl values are not comparable with the paper's figures"}
    fit.close()
    plan.close()
    return out


def bench_served_loop(pkg, torch, dev, telescopes=4, frames=60, gain=0.4, fit_iters=4):
    """Closed loop through the server (Algorithm 4.1 per telescope): `telescopes` E-ELT systems
    with their three mirrors, admitted with tomo_server_admit_loop (cluster size 4).  Each has
    its own frozen-flow atmosphere and a plant on the GPU (the library's own measurement minus
    its mirror slopes of the commands returned two frames earlier, plus seeded noise).  A round
    submits every telescope's residual frame from pinned host memory and waits for the
    commands; the rounds run as fast as the loop closes, with no pacing.  Reported: control
    steps per second over all telescopes, the server's submit-to-result latency, and the
    long-exposure Strehl at 2200 nm over the second half of the frames."""
    from synth import configs, FrozenFlow, gaussian_noise
    g = configs.with_fitting(configs.config1())
    srv = pkg.Server(iters=int(g["iters"]), max_in_flight=4, queue_depth=4, result_slots=8)
    ids = [srv.admit_loop(g, gain=gain, fit_iters=fit_iters, cluster_size=4) for _ in range(telescopes)]
    plant = pkg.Plan(g)
    pfit = pkg.Fit(plant, g["fitting"])
    n, ns, na, nd = plant.n, plant.n_slopes, pfit.n, int(pfit.info.n_dir)
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in g["wfs"]])
    truth = torch.empty((telescopes, frames, n), dtype=torch.float32, device=dev)
    meas = torch.empty((telescopes, frames, ns), dtype=torch.float32, device=dev)
    for i in range(telescopes):
        flow = FrozenFlow(g, 1, instance=20 + i)
        for t in range(frames):
            truth[i, t].copy_(torch.from_numpy(np.concatenate([p.ravel() for p in flow.layers(0.002 * t)])
                                               .astype(np.float32)))
            plant.layers_to_slopes(truth[i, t], meas[i, t])
            meas[i, t] += torch.from_numpy((gaussian_noise(ns, 1.0, 7_000_000 + 1000 * i + t) * sig)
                                           .astype(np.float32)).to(dev)
    hist = [[torch.zeros(na, dtype=torch.float32, device=dev) for _ in range(2)] for _ in range(telescopes)]
    s_dev = torch.empty(ns, dtype=torch.float32, device=dev)
    s_host = [torch.empty(ns, dtype=torch.float32, pin_memory=True) for _ in range(telescopes)]
    rms = torch.empty((telescopes, frames, nd), dtype=torch.float64, device=dev)
    lat, t0 = [], None
    for t in range(frames):
        if t == 2:
            torch.cuda.synchronize()
            t0 = time.perf_counter()   # from the first frame that closes the loop
        for i, tid in enumerate(ids):
            a_applied = hist[i][t]     # the commands returned two frames earlier
            pfit.residual_rms(truth[i, t], a_applied, rms[i, t])
            pfit.mirror_slopes(a_applied, s_dev, slopes_in=meas[i, t], scale=-1.0)
            s_host[i].copy_(s_dev)
            assert srv.submit(tid, s_host[i].numpy(), tag=t)
        got = 0
        while got < telescopes:
            for r in srv.poll():
                assert r["status"] == 0
                i = ids.index(r["telescope"])
                a = srv.result(r["telescope"], r["result_slot"], r["tag"])
                hist[i].append(torch.from_numpy(a).to(dev))
                if t >= 2:
                    lat.append(1000.0 * (r["t_done"] - r["t_submit"]))
                got += 1
            if got < telescopes:
                time.sleep(0.0001)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    le = slice(frames // 2, frames)
    strehl = np.exp(-(rms.cpu().numpy()[:, le] * (500.0 / 2200.0)) ** 2).mean(axis=1)   # [telescope, direction]
    out = {"telescopes": telescopes, "frames_per_telescope": frames, "gain": gain, "fit_iters": fit_iters,
           "cluster_size": 4, "max_in_flight": 4,
           "control_steps_per_s": telescopes * (frames - 2) / wall,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "launches": stats["launches"],
           "strehl_2200nm_long_exposure_field_average": [float(x) for x in strehl.mean(axis=1)],
           "note": "rounds of one frame per telescope, each waiting for the commands that close the loop; "
                   "the plant (measurement, mirror slopes, Strehl) runs on the same GPU between the rounds"}
    pfit.close()
    plant.close()
    return out


def served_geometries():
    """16 telescopes cycling the three geometry families: the 8 m system (FP32 operator, Jacobi
    PCG), the E-ELT system, and instances of the uneven 64-instance set."""
    from synth import configs
    uneven = configs.config2()
    out = []
    for i in range(16):
        if i % 3 == 0:
            g = configs.config0()
            g = dict(g, precision=0, precond=1, iters=10, name=g["name"].replace("fp64", "fp32-pcg"))
        elif i % 3 == 1:
            g = configs.config1()
        else:
            g = uneven[i]
        out.append(g)
    return out


def bench_served(pkg, torch, args, dev, frames_per_tel=16, rate_hz=500.0):
    """Served stream: every telescope emits frames at rate_hz with a seeded phase for
    args.serve_seconds; the server solves each warm-started (10 PCG iterations), batching the
    frames that wait.  Latency is from tomo_server_submit to the coefficients in host memory."""
    from synth import FrozenFlow, gaussian_noise
    geoms = served_geometries()
    # frames: frozen-flow screens measured by a temporary plan, plus noise (host float32)
    frames = []
    for i, g in enumerate(geoms):
        p = pkg.Plan(g)
        flow = FrozenFlow(g, 3, instance=i)
        sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                              for w in g["wfs"]])
        lay = torch.empty(p.n, dtype=torch.float32, device=dev)
        sl = torch.empty(p.n_slopes, dtype=torch.float32, device=dev)
        fr = []
        for k in range(frames_per_tel):
            lay.copy_(torch.from_numpy(np.concatenate([x.ravel() for x in flow.layers(k / rate_hz)])
                                       .astype(np.float32)))
            p.layers_to_slopes(lay, sl)
            noise = gaussian_noise(p.n_slopes, 1.0, 5_000_000 + 1000 * i + k) * sig
            fr.append(np.ascontiguousarray(sl.cpu().numpy() + noise.astype(np.float32)))
        frames.append(fr)
        p.close()
    from paper_1302_3734_gb300.autotune import tune
    (c_s, tf_s), tab_s = tune(geoms, 10)
    srv = pkg.Server(budget_bytes=16 << 30, iters=10, max_in_flight=4, queue_depth=64, result_slots=2)
    srv.set_policy(latest_only=True)
    ids = []
    for g in geoms:
        cc = c_s
        while True:
            try:
                ids.append(srv.admit(g, cluster_size=cc, transforms=tf_s))
                break
            except pkg.TomoError as e:
                if e.status not in (1, 8) or cc >= 16:
                    raise
                cc *= 2
    stats0 = srv.stats()
    # warm-up: every telescope's first frame, so the batch graphs exist
    for i, t in enumerate(ids):
        srv.submit(t, frames[i][0], tag=-1)
    srv.drain(120.0)
    srv.poll()

    def stream(rate, seconds, seed):
        """Every telescope submits frames at `rate` Hz (seeded phases) for `seconds`."""
        period = 1.0 / rate
        n_frames = int(seconds * rate)
        phase = np.random.default_rng(seed).uniform(0.0, period, len(ids))
        launches0 = srv.stats()["launches"]
        t0 = srv.clock() + 0.05
        sched = sorted((t0 + phase[i] + k * period, i, k) for i in range(len(ids)) for k in range(n_frames))
        results, lag, full = [], [], 0
        j = 0
        while j < len(sched):
            now = srv.clock()
            if sched[j][0] > now:
                if sched[j][0] - now > 0.0005:
                    results += srv.poll()
                    time.sleep(0.0002)
                continue
            while j < len(sched) and sched[j][0] <= now:
                ts, i, k = sched[j]
                if not srv.submit(ids[i], frames[i][k % frames_per_tel], tag=k):
                    full += 1
                lag.append(now - ts)
                j += 1
        srv.drain(300.0)
        results += srv.poll()
        ok = [r for r in results if r["status"] == 0]
        lat = np.array([r["t_done"] - r["t_submit"] for r in ok]) * 1000.0
        span = max(r["t_done"] for r in ok) - t0
        return sched, ok, results, lat, span, lag, full, srv.stats()["launches"] - launches0

    # capacity curve: shorter streams at lower offered loads
    curve = []
    for rate in (250.0, 350.0, 425.0, 475.0):
        sched, ok, results, lat, span, _, _, nl = stream(rate, 2.0, 7)
        curve.append({"offered_frames_per_s": len(ids) * rate, "solves_per_s": len(ok) / span,
                      "superseded_fraction": sum(1 for r in results if r["status"] == 10) / len(sched),
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "mean_frames_per_launch": len(ok) / max(1, nl)})
    sched, ok, results, lat, span, lag, full, nl = stream(rate_hz, args.serve_seconds, 3)
    srv.close()
    superseded = sum(1 for r in results if r["status"] == 10)
    curve.append({"offered_frames_per_s": len(ids) * rate_hz, "solves_per_s": len(ok) / span,
                  "superseded_fraction": superseded / len(sched),
                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                  "mean_frames_per_launch": len(ok) / max(1, nl)})
    kinds = {}
    for r in ok:
        name = geoms[ids.index(r["telescope"])]["name"].split("-")[0]
        kinds.setdefault(name, []).append((r["t_done"] - r["t_submit"]) * 1000.0)
    return {
        "telescopes": len(ids), "rate_hz_per_telescope": rate_hz, "seconds": args.serve_seconds,
        "frames_offered": len(sched), "frames_done": len(ok), "frames_refused_queue_full": full,
        "frames_superseded": superseded, "policy": "latest frame (older waiting frames superseded)",
        "cluster_size": c_s, "transforms": "streamed" if tf_s == 2 else "cluster",
        "autotune_solves_per_s": tab_s,
        "solves_per_s": len(ok) / span,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "latency_ms_p99_by_family": {k: float(np.percentile(v, 99)) for k, v in kinds.items()},
        "launches": nl, "mean_frames_per_launch": len(ok) / max(1, nl),
        "capacity_curve": curve,
        "client_pacing_lag_ms_p99": float(np.percentile(np.array(lag) * 1000.0, 99)),
        "device_bytes_admitted": stats0["bytes_in_use"], "budget_bytes": stats0["budget_bytes"],
        "workload": "16 telescopes cycling the 8 m (FP32 PCG), E-ELT and uneven-instance "
                    "geometries; 500 Hz frozen-flow frames each; 10 PCG iterations, warm start; "
                    "capacity curve: 2 s streams at 250-475 Hz per telescope, then the 500 Hz stream",
    }


def profile_leg(args):
    """One workload's solves and nothing else, so a profiler's launch list holds only them:
    eelt (the E-ELT frame, 10 warm PCG iterations, graph), batch16 (16 E-ELT instances at
    cluster size 2, streamed transforms), uneven64 (the 64 uneven instances at cluster size 4,
    streamed transforms), large (the 100 m system, 20 cold PCG iterations).  The batches take
    the autotuner's pick of the batched legs.  Plans are built before the first solve."""
    import torch
    import paper_1302_3734_gb300 as pkg
    from paper_1302_3734_gb300 import build
    from synth import configs, gaussian_noise
    build.build()
    dev = torch.device("cuda", 0)
    leg = args.profile_leg
    tf = 0
    if leg == "large":
        geoms, C, iters, warm = [configs.config4()], 0, 20, False
    elif leg == "uneven64":
        geoms, C, iters, warm, tf = configs.config2(), 4, 10, True, 2
    else:
        geoms, C, iters, warm = [configs.config1()] * (16 if leg == "batch16" else 1), (2 if leg == "batch16" else 0), 10, True
        tf = 2 if leg == "batch16" else 0
    plans = []
    for g in geoms:
        cc = C
        while True:
            try:
                plans.append(pkg.Plan(g, cluster_size=cc, transforms=tf))
                break
            except pkg.TomoError as e:
                if e.status not in (1, 8) or cc == 0 or cc >= 16:
                    raise
                cc *= 2
    sl = [torch.tensor(gaussian_noise(p.n_slopes, 0.3, 100 + i), dtype=torch.float32, device=dev)
          for i, p in enumerate(plans)]
    xs = [torch.zeros(p.n, dtype=torch.float32, device=dev) for p in plans]
    for _ in range(args.solves):
        if len(plans) == 1:
            plans[0].solve(sl[0], xs[0], iters, warm=warm)
        else:
            pkg.solve_batch(plans, sl, xs, iters, warm=warm)
    torch.cuda.synchronize()
    print(f"{leg}: {args.solves} solves of {len(plans)} plan(s), {iters} PCG iterations", flush=True)
    for p in plans:
        p.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_leg:
        return profile_leg(args)
    import torch
    import paper_1302_3734_gb300 as pkg
    from paper_1302_3734_gb300 import build
    from synth import gaussian_noise

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    geom, cfg = workload()
    dev = torch.device("cuda", local)
    plan = pkg.Plan(geom)
    info = plan.info
    n, ns = plan.n, plan.n_slopes
    F = args.warmup + args.steps
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in geom["wfs"]])

    # frames: noise-free slopes from the library's measurement of the screens + noise
    layers = torch.empty(n, dtype=torch.float32, device=dev)
    slopes = torch.empty((F, ns), dtype=torch.float32, device=dev)
    for k in range(F):
        phis = frame_screens(geom, k, rank)
        layers.copy_(torch.from_numpy(np.concatenate([p.ravel() for p in phis]).astype(np.float32)))
        plan.layers_to_slopes(layers, slopes[k])
        noise = gaussian_noise(ns, 1.0, 1_000_000 + 1000 * rank + k)
        slopes[k] += torch.from_numpy((noise * sig).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    x = torch.zeros(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    iters = int(geom["iters"])

    def run(use_graphs, steps, first, record):
        plan.set_launch_mode(use_graphs)
        times = []
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.solve(slopes[(first + k) % F], x, iters, warm=True)
            e1.record()
            if record:
                times.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    # warm-up (also builds the CUDA graph), then the timed region
    run(1, args.warmup, 0, False)
    # plain one-launch-per-kernel PCG on the same frames, for comparison
    plain = run(0, min(args.steps, 50), 0, True)
    x.zero_()
    run(1, args.warmup, 0, False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    with Clocks(local) as clk:
        times = run(1, args.steps, args.warmup, True)
    launches = pkg.launch_count() - launches0
    if dist:
        dist.barrier()
    tot_ms = max_over_ranks(sum(times), dist, dev)
    value = job_rate(ws, args.steps, tot_ms)
    ms_step = tot_ms / args.steps

    # end to end through the public API: pinned host slopes in, coefficients out.
    # Every frame has its own pinned buffer (no host write races an earlier
    # asynchronous copy), and untimed warm-up steps build the graph that the
    # device input buffer selects.
    host_frames = slopes.cpu().pin_memory()
    h_x = torch.empty(n, dtype=torch.float32, pin_memory=True)
    d_s = torch.empty(ns, dtype=torch.float32, device=dev)

    def run_e2e(steps, first, record):
        out = []
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            d_s.copy_(host_frames[(first + k) % F], non_blocking=True)
            plan.solve(d_s, x, iters, warm=True)
            h_x.copy_(x, non_blocking=True)
            e1.record()
            if record:
                out.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in out]

    run_e2e(args.warmup, 0, False)
    e2e_ms = run_e2e(args.steps, args.warmup, True)

    # per-kernel times (events around every launch, direct launches)
    plan.set_kernel_timing(True)
    run(0, min(args.steps, 50), args.warmup, False)
    kt = plan.kernel_times()
    plan.set_kernel_timing(False)
    per_launch_bytes = launch_bytes([plan], [geom])
    dominant = max((k for k in per_launch_bytes if kt[k][0] > 0), key=lambda k: kt[k][1])
    cnt, ms = kt[dominant]
    achieved = per_launch_bytes[dominant] * cnt / (ms / 1000.0) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    l2_gbs = l2_probe(pkg, torch, dev)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(cfg, l2="flushed (256 MiB write) before every timed step",
                       parallelism=f"replicas x{ws}" if ws > 1 else "single GPU",
                       launch="CUDA graph of the whole frame"),
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
        "plain_launch": {"value": 1000.0 / float(np.mean(plain)), "unit": "solves/s",
                         "p50_ms": float(np.percentile(plain, 50)),
                         "p99_ms": float(np.percentile(plain, 99)),
                         "note": "same kernels, one launch per kernel, no graph"},
        "e2e": {"value": ws * 1000.0 / float(np.mean(e2e_ms)), "unit": "solves/s",
                "h2d_bytes_per_step": 4 * ns, "d2h_bytes_per_step": 4 * n,
                "p99_ms": float(np.percentile(e2e_ms, 99))},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": ncu_traffic(dominant),
                     "peak_source": peak_src,
                     "l2_peak_gbs": l2_gbs, "frac_of_l2_peak": achieved / l2_gbs,
                     "bytes_per_launch": per_launch_bytes[dominant],
                     "kernel_ms_per_launch": {k: v[1] / v[0] for k, v in kt.items() if v[0]},
                     "bytes_per_iteration": info.bytes_per_iteration},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_batch:
        line["batched"] = bench_batched(pkg, torch, geom, slopes, flush, iters, args, peak, dev)
    if not args.no_large and rank == 0:
        line["large"] = bench_large(pkg, torch, dev, flush, peak)
    if not args.no_loop and rank == 0:
        line["closed_loop"] = bench_closed_loop(pkg, torch, dev, flush, args.loop_frames)
    if args.serve_seconds > 0 and rank == 0:
        line["served"] = bench_served(pkg, torch, args, dev)
    if not args.no_loop and args.serve_seconds > 0 and rank == 0:
        line["served_closed_loop"] = bench_served_loop(pkg, torch, dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import Tomography
        ora = Tomography(geom)
        frames = [ora.measure(frame_screens(geom, k, 0)) + gaussian_noise(ns, 1.0, 1_000_000 + k) * sig
                  for k in range(min(F, 20))]
        line["cpu_baseline"] = cpu_baseline(geom, frames, np.zeros(n), args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
