"""Launch-shape autotuner for batched solves.

Two knobs set how a plan's kernels are shaped:

* the cluster size C (``cluster_size``): the cluster transform kernels run one
  thread-block cluster of C CTAs per layer, and the gather works on bands of
  N/C rows.  A large C finishes one solve soonest (a layer's rows spread over
  more SMs); many instances solved together fill the GPU anyway, and then a
  small C wins: fewer cluster barriers per level, more clusters resident;
* the transforms (``transforms``): cluster kernels with the gather staged in
  the analysis kernel when its tables fit (1), or streamed level passes over
  row tiles with the gather in its own kernel (2).

Which shape is best depends on the geometries, the batch and the GPU, so it is
measured: every candidate builds the batch's plans, times ``solve_batch`` with
CUDA events, and the fastest wins.  Results are cached per (batch signature,
iterations, device) in memory and, when a path is given, in a JSON file.
"""
import hashlib
import json
import os

import numpy as np

from .binding import Plan, TomoError, solve_batch

CANDIDATES = (16, 8, 4, 2, 1)
TRANSFORMS = (1, 2)     # cluster kernels, streamed passes
_cache = {}


def signature(geoms, iters):
    """Hash of what decides the launch shape: layer grids, sensors, wavelet, precision."""
    h = hashlib.sha256()
    for g in geoms:
        h.update(json.dumps({
            "layers": [(int(l["N"]), float(l["altitude"])) for l in g["layers"]],
            "wfs": [(int(w["n_sub"]), float(w["height"]), bool(w["tt_only"])) for w in g["wfs"]],
            "wavelet": (int(g["wavelet_order"]), int(g["levels"])),
            "precision": int(g["precision"]), "precond": int(g["precond"]),
        }, sort_keys=True).encode())
    h.update(str((len(geoms), int(iters))).encode())
    return h.hexdigest()[:24]


def _plans(geoms, c, transforms=0):
    """Plans at cluster size c; a plan that cannot take c gets the next larger size."""
    plans = []
    try:
        for g in geoms:
            cc, p = c, None
            while p is None:
                try:
                    p = Plan(g, cluster_size=cc, transforms=transforms)
                except TomoError as e:
                    if e.status not in (1, 8) or cc >= 16:
                        raise
                    cc *= 2
            plans.append(p)
        return plans
    except TomoError:
        for p in plans:
            p.close()
        return None


def _time(torch, plans, iters, steps, warmup):
    dev = torch.device("cuda")
    rng = np.random.default_rng(0)
    sl, xs = [], []
    for p in plans:
        dt = torch.float64 if p.precision else torch.float32
        sl.append(torch.tensor(rng.standard_normal(p.n_slopes) * 0.3, dtype=dt, device=dev))
        xs.append(torch.zeros(p.n, dtype=dt, device=dev))
    for _ in range(warmup):
        solve_batch(plans, sl, xs, iters)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        solve_batch(plans, sl, xs, iters)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_cluster_size(geoms, iters=10, candidates=CANDIDATES, steps=10, warmup=3, path=None):
    """Best cluster size for solving `geoms` together.  Returns (C, table) where table maps
    each candidate to its measured solves/s (None: no plan could be built)."""
    import torch
    key = f"{signature(geoms, iters)}:{torch.cuda.get_device_name()}"
    if key in _cache:
        return _cache[key]
    if path and os.path.exists(path):
        try:
            stored = json.load(open(path))
            if key in stored:
                c, table = stored[key]["best"], {int(k): v for k, v in stored[key]["table"].items()}
                _cache[key] = (c, table)
                return c, table
        except (OSError, ValueError, KeyError):
            pass
    table = {}
    for c in candidates:
        plans = _plans(geoms, c)
        if plans is None:
            table[c] = None
            continue
        ms = _time(torch, plans, iters, steps, warmup)
        table[c] = len(geoms) * 1000.0 / ms
        for p in plans:
            p.close()
    valid = {c: v for c, v in table.items() if v is not None}
    if not valid:
        raise RuntimeError("no candidate cluster size can build these plans")
    best = max(valid, key=valid.get)
    _cache[key] = (best, table)
    if path:
        try:
            stored = json.load(open(path)) if os.path.exists(path) else {}
        except (OSError, ValueError):
            stored = {}
        stored[key] = {"best": best, "table": {str(k): v for k, v in table.items()}}
        with open(path, "w") as f:
            json.dump(stored, f, indent=1)
    return best, table


def tune(geoms, iters=10, candidates=CANDIDATES, transforms=TRANSFORMS, steps=10, warmup=3):
    """Best (cluster size, transforms) for solving `geoms` together.  Returns ((C, tf), table)
    where table maps "C/tf" to the measured solves/s (None: no plan could be built)."""
    import torch
    key = f"shape:{signature(geoms, iters)}:{torch.cuda.get_device_name()}"
    if key in _cache:
        return _cache[key]
    table = {}
    for c in candidates:
        for tf in transforms:
            plans = _plans(geoms, c, tf)
            if plans is None:
                table[f"{c}/{tf}"] = None
                continue
            ms = _time(torch, plans, iters, steps, warmup)
            table[f"{c}/{tf}"] = len(geoms) * 1000.0 / ms
            for p in plans:
                p.close()
    valid = {k: v for k, v in table.items() if v is not None}
    if not valid:
        raise RuntimeError("no candidate launch shape can build these plans")
    best = max(valid, key=valid.get)
    c, tf = (int(x) for x in best.split("/"))
    _cache[key] = ((c, tf), table)
    return (c, tf), table
