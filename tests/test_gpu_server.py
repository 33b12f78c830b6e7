"""The served stream (tomo_server_*): frames of several telescopes of different
sizes, admitted by memory, solved warm-started and batched on arrival.

* every frame served in the mix is bitwise the frame solved alone (the same
  telescope's frames through tomo_solve, one after the other, warm-started);
* sampled frames match the FP64 oracle (PCG from the server's own previous
  frame, as a warm start is defined);
* admission by a device-memory budget, release, the bounded frame queue and
  drain.
"""

import time

import numpy as np
import pytest

from oracle import Tomography
from synth import configs, FrozenFlow, gaussian_noise

from test_gpu_parity import ERRORS, error_log, rel  # noqa: F401  (shared error log)

pytestmark = pytest.mark.gpu

ITERS = 6


def _geoms():
    small = configs.small_lgs_config(16, 32, 3, 2)
    ragged = configs.small_lgs_config(24, 64, 2, 3, order=2)
    cfg0 = configs.config0()
    cfg0 = dict(cfg0, precision=0, precond=1, name=cfg0["name"].replace("fp64", "fp32-pcg"))
    return [small, ragged, cfg0]


def _frames(geom, k_frames, seed):
    ora = Tomography(geom)
    ns = int(ora.meas_offsets[-1])
    sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"])
                          for w in geom["wfs"]])
    flow = FrozenFlow(geom, 3, instance=seed)
    out = []
    for k in range(k_frames):
        s = ora.measure(flow.layers(0.002 * k)) + gaussian_noise(ns, 1.0, 50_000 + 100 * seed + k) * sig
        out.append(np.ascontiguousarray(s, dtype=np.float32))
    return ora, out


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1302_3734_gb300 import build
    build.build()
    import paper_1302_3734_gb300 as pkg
    return torch, pkg


def _serve(pkg, geoms, frames, shape=None, **kw):
    srv = pkg.Server(iters=ITERS, result_slots=len(frames[0]) + 1, queue_depth=len(frames[0]) + 1, **kw)
    ids = [srv.admit(g) if shape is None else srv.admit(g, cluster_size=shape[0], transforms=shape[1])
           for g in geoms]
    # interleaved arrivals, as several telescopes emit frames at the same rate
    for k in range(len(frames[0])):
        for i, tid in enumerate(ids):
            assert srv.submit(tid, frames[i][k], tag=k)
    srv.drain(120.0)
    res = srv.poll()
    got = {}
    for r in res:
        assert r["status"] == 0
        assert r["t_submit"] <= r["t_launch"] <= r["t_done"]
        x = srv.result(r["telescope"], r["result_slot"], r["tag"])
        assert x is not None
        got[(ids.index(r["telescope"]), r["tag"])] = x
    stats = srv.stats()
    srv.close()
    return got, res, stats


@pytest.mark.parametrize("shape", [None, (4, 2)], ids=["default", "C4-streamed"])
def test_served_frames_are_bitwise_the_frames_solved_alone(lib, shape):
    """Every served frame equals the same frame solved alone by a plan of the same
    launch shape: the default shapes, and the streamed transforms at cluster size 4
    that the served benchmark's autotuner picks."""
    torch, pkg = lib
    geoms = _geoms()
    K = 5
    data = [_frames(g, K, i) for i, g in enumerate(geoms)]
    frames = [d[1] for d in data]
    got, res, stats = _serve(pkg, geoms, frames, shape=shape, max_in_flight=2)
    assert stats["frames_done"] == K * len(geoms)
    assert max(r["batch_size"] for r in res) > 1, "frames of different telescopes never shared a launch"
    for i, g in enumerate(geoms):
        plan = pkg.Plan(g) if shape is None else pkg.Plan(g, cluster_size=shape[0], transforms=shape[1])
        x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
        for k in range(K):
            s = torch.tensor(frames[i][k], device="cuda")
            plan.solve(s, x, ITERS, warm=True)
            alone = x.cpu().numpy()
            assert np.array_equal(alone, got[(i, k)]), (g["name"], k)
        plan.close()


def test_served_frames_match_the_oracle(lib):
    torch, pkg = lib
    geoms = _geoms()
    K = 4
    data = [_frames(g, K, 10 + i) for i, g in enumerate(geoms)]
    got, _, _ = _serve(pkg, geoms, [d[1] for d in data], max_in_flight=3)
    for i, g in enumerate(geoms):
        ora = data[i][0]
        for k in (0, K - 1):
            x0 = np.zeros(ora.n) if k == 0 else got[(i, k - 1)].astype(np.float64)
            s = data[i][1][k].astype(np.float64)
            x_ref = ora.pcg(ora.rhs(s), x0, ITERS, ora.jacobi_diagonal() if g["precond"] else None)
            e = rel(ora.join(ora.synthesis(got[(i, k)].astype(np.float64))),
                    ora.join(ora.synthesis(x_ref)), f"served/{g['name']}/frame{k}")
            assert e < 1e-5, (g["name"], k, e)


def test_served_breakdown_is_the_frame_status(lib):
    """A frame of NaN slopes comes back with TOMO_ERR_BREAKDOWN; the telescope's
    warm start stays that of its previous frame, so its next frame is served as
    if the broken one had not been there, and the other telescope is unaffected."""
    torch, pkg = lib
    geoms = _geoms()[:2]
    K = 3
    frames = [_frames(g, K, 30 + i)[1] for i, g in enumerate(geoms)]
    srv = pkg.Server(iters=ITERS, result_slots=8, queue_depth=8)
    ids = [srv.admit(g) for g in geoms]
    nan = np.full_like(frames[0][0], np.nan)
    order = [(0, frames[0][0], 0), (1, frames[1][0], 0), (0, nan, 1), (1, frames[1][1], 1),
             (0, frames[0][1], 2), (1, frames[1][2], 2)]
    for i, s, tag in order:
        assert srv.submit(ids[i], s, tag=tag)
        srv.drain(60.0)                        # one frame at a time: a fixed order
    res = {(ids.index(r["telescope"]), r["tag"]): r for r in srv.poll()}
    assert res[(0, 1)]["status"] == 7
    assert all(r["status"] == 0 for key, r in res.items() if key != (0, 1))
    got0 = srv.result(ids[0], res[(0, 2)]["result_slot"], 2)
    got1 = srv.result(ids[1], res[(1, 2)]["result_slot"], 2)
    srv.close()
    for i, ks, got in ((0, (0, 1), got0), (1, (0, 1, 2), got1)):
        plan = pkg.Plan(geoms[i])
        x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
        for k in ks:
            plan.solve(torch.tensor(frames[i][k], device="cuda"), x, ITERS, warm=True)
        assert np.array_equal(x.cpu().numpy(), got), i
        plan.close()


def test_admission_by_memory_budget(lib):
    torch, pkg = lib
    g = configs.small_lgs_config(16, 32, 3, 2)
    probe = pkg.Server(iters=2)
    a = probe.admit(g)
    one = probe.stats()["bytes_in_use"]
    probe.close()
    srv = pkg.Server(budget_bytes=int(2.5 * one), iters=2)
    ids = [srv.admit(g), srv.admit(g)]
    with pytest.raises(pkg.TomoError) as ei:
        srv.admit(g)
    assert ei.value.status == 4
    assert srv.stats()["telescopes"] == 2
    srv.release(ids[0])
    ids.append(srv.admit(g))
    assert srv.stats()["telescopes"] == 2 and srv.stats()["bytes_in_use"] <= int(2.5 * one)
    s = np.zeros(srv.info(ids[-1]).n_slopes, dtype=np.float32)
    assert srv.submit(ids[-1], s, tag=7)
    srv.drain(60.0)
    (r,) = srv.poll()
    assert r["tag"] == 7 and r["status"] == 0
    assert np.all(srv.result(ids[-1], r["result_slot"], 7) == 0.0)   # zero data, zero start: x = 0
    srv.close()
    del a


def test_bounded_queue_release_and_drain(lib):
    torch, pkg = lib
    g = configs.small_lgs_config(16, 32, 3, 2)
    srv = pkg.Server(iters=400, queue_depth=2, result_slots=2)
    tid = srv.admit(g)
    s = np.ones(srv.info(tid).n_slopes, dtype=np.float32)
    ok = [srv.submit(tid, s, tag=k) for k in range(6)]
    assert ok[:2] == [True, True] and not all(ok), ok   # the first frame holds a slot while it runs
    srv.drain(60.0)
    assert all(r["status"] == 0 for r in srv.poll())
    # frames still waiting when their telescope leaves are dropped; drain still returns
    t2 = srv.admit(g)
    for k in range(2):
        srv.submit(t2, s, tag=100 + k)
    srv.release(t2)
    srv.drain(60.0)
    srv.poll()
    assert srv.stats()["telescopes"] == 1
    srv.close()


def test_latest_frame_policy_supersedes_stale_frames(lib):
    torch, pkg = lib
    g = configs.small_lgs_config(16, 32, 3, 2)
    srv = pkg.Server(iters=3000, queue_depth=8, result_slots=4)
    srv.set_policy(latest_only=True)
    tid = srv.admit(g)
    s = np.ones(srv.info(tid).n_slopes, dtype=np.float32)
    assert srv.submit(tid, s, tag=0)
    t0 = time.monotonic()
    while srv.stats()["in_flight"] == 0 and time.monotonic() - t0 < 5.0:
        time.sleep(0.0005)
    assert srv.stats()["in_flight"] == 1   # frame 0 runs (3000 iterations); 1..4 wait behind it
    for k in range(1, 5):
        assert srv.submit(tid, s, tag=k)
    srv.drain(60.0)
    res = {r["tag"]: r for r in srv.poll()}
    assert res[0]["status"] == 0 and res[4]["status"] == 0      # the running frame and the newest
    assert [res[k]["status"] for k in (1, 2, 3)] == [10, 10, 10]  # superseded
    assert srv.stats()["frames_superseded"] == 3
    srv.close()


def test_every_100th_frame_of_a_served_stream_matches_the_oracle(lib):
    torch, pkg = lib
    geoms = _geoms()[:2]
    K = 201
    data = [_frames(g, K, 20 + i) for i, g in enumerate(geoms)]
    srv = pkg.Server(iters=ITERS, queue_depth=256, result_slots=256)
    ids = [srv.admit(g) for g in geoms]
    for k in range(K):
        for i, tid in enumerate(ids):
            assert srv.submit(tid, data[i][1][k], tag=k)
    srv.drain(300.0)
    res = srv.poll()
    assert len(res) == K * len(ids) and all(r["status"] == 0 for r in res)
    got = {(ids.index(r["telescope"]), r["tag"]): srv.result(r["telescope"], r["result_slot"], r["tag"])
           for r in res if r["tag"] % 100 in (0, 99)}
    srv.close()
    for i, g in enumerate(geoms):
        ora = data[i][0]
        for k in (100, 200):
            x0 = got[(i, k - 1)].astype(np.float64)
            s = data[i][1][k].astype(np.float64)
            x_ref = ora.pcg(ora.rhs(s), x0, ITERS, ora.jacobi_diagonal())
            e = rel(got[(i, k)].astype(np.float64), x_ref, f"served-stream/{g['name']}/frame{k}")
            assert e < 1e-5, (g["name"], k, e)


def test_closed_loop_telescopes_are_their_control_steps_and_match_the_oracle_loop(lib):
    """Two telescopes served in closed loop (Algorithm 4.1, gain 0.4, two-frame delay) next to
    an open-loop one.  A CPU plant measures each frozen-flow atmosphere behind the commands
    the server returned two frames earlier.  The served commands are bitwise the control
    steps run directly through the Fit API on the same residual slopes, and follow the
    oracle's own closed loop."""
    from oracle.control import Control
    torch, pkg = lib
    loop_geoms = [configs.with_fitting(configs.small_lgs_config(16, 32, 3, 2), altitudes=(0.0, 4000.0, 9000.0),
                                       field_arcmin=1.2, n_dir=3),
                  configs.with_fitting(configs.small_lgs_config(24, 64, 2, 3, order=2), altitudes=(0.0, 6000.0),
                                       field_arcmin=1.2, n_dir=3)]
    gain, fit_iters, K = 0.4, 4, 6
    srv = pkg.Server(iters=ITERS, queue_depth=4, result_slots=8)
    ids = [srv.admit_loop(g, gain=gain, fit_iters=fit_iters) for g in loop_geoms]
    open_geom = configs.small_lgs_config(16, 32, 3, 2)
    open_id = srv.admit(open_geom)
    _, open_frames = _frames(open_geom, K, 5)
    ctls = [Control(g) for g in loop_geoms]
    meas = []
    for i, (g, ctl) in enumerate(zip(loop_geoms, ctls)):
        ns = int(ctl.tom.meas_offsets[-1])
        sig = np.concatenate([np.full(2 if w["tt_only"] else 2 * int(w["valid"].sum()), w["sigma"]) for w in g["wfs"]])
        flow = FrozenFlow(g, 3, instance=30 + i)
        meas.append([ctl.tom.measure(flow.layers(0.002 * t)) + gaussian_noise(ns, 1.0, 800 + 50 * i + t) * sig
                     for t in range(K)])
    served = [[np.zeros(c.fit.n), np.zeros(c.fit.n)] for c in ctls]   # a_0 = a_1 = 0
    submitted = [[] for _ in ctls]
    for t in range(K):
        for i, tid in enumerate(ids):
            s = (meas[i][t] - ctls[i].mirror_slopes(served[i][t].astype(np.float64))).astype(np.float32)
            submitted[i].append(s)
            assert srv.submit(tid, s, tag=t)
        assert srv.submit(open_id, open_frames[t], tag=t)
        srv.drain(60.0)
        for r in srv.poll():
            assert r["status"] == 0 and r["tag"] == t
            if r["telescope"] in ids:
                served[ids.index(r["telescope"])].append(srv.result(r["telescope"], r["result_slot"], t))
    srv.close()
    for i, g in enumerate(loop_geoms):
        # the same control steps through the Fit API
        plan = pkg.Plan(g)
        fit = pkg.Fit(plan, g["fitting"])
        buf = [torch.zeros(fit.n, dtype=torch.float32, device="cuda") for _ in range(2)]
        x = torch.zeros(plan.n, dtype=torch.float32, device="cuda")
        rec = torch.zeros(fit.n, dtype=torch.float32, device="cuda")
        for t in range(K):
            a_tm2, a_tm1 = buf[t % 2], buf[(t + 1) % 2]
            fit.polc_step(torch.tensor(submitted[i][t], device="cuda"), x, rec, a_tm2, a_tm1, a_tm2, gain, ITERS,
                          fit_iters, warm=True)
            assert np.array_equal(a_tm2.cpu().numpy(), served[i][t + 2]), (g["name"], t)
        fit.close()
        plan.close()
        # the oracle's closed loop on the same measurements
        ctl = ctls[i]
        a = [np.zeros(ctl.fit.n), np.zeros(ctl.fit.n)]
        xo, reco = np.zeros(ctl.tom.n), np.zeros(ctl.fit.n)
        for t in range(K):
            a_t, xo, reco = ctl.step(meas[i][t] - ctl.mirror_slopes(a[t]), a[t], a[t + 1], xo, reco, gain,
                                     ITERS, fit_iters)
            a.append(a_t)
            e = rel(served[i][t + 2].astype(np.float64), a_t, f"served-closed-loop/{g['name']}/frame{t}")
            assert e < 1e-5, (g["name"], t, e)


def test_drain_deadline_reports_a_timeout_and_the_server_stays_usable(lib):
    torch, pkg = lib
    g = configs.small_lgs_config(16, 32, 3, 2)
    srv = pkg.Server(iters=3000, queue_depth=2, result_slots=2)
    tid = srv.admit(g)
    s = np.ones(srv.info(tid).n_slopes, dtype=np.float32)
    assert srv.submit(tid, s, tag=1)
    with pytest.raises(pkg.TomoError) as ei:
        srv.drain(1e-4)                     # a 3000-iteration frame is still on the GPU
    assert ei.value.status == 6
    srv.drain(60.0)
    (r,) = srv.poll()
    assert r["status"] == 0 and r["tag"] == 1
    assert srv.submit(tid, s, tag=2)
    srv.drain(60.0)
    assert [r["tag"] for r in srv.poll()] == [2]
    srv.close()
