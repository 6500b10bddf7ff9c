"""Benchmark of the B300 acoustic FD propagator (one JSON line on stdout).

Workload: the layered 3D single-shot stencil, 512^3 FP32 grid, radius-4
Laplacian, 20-point sponge on all faces, 10 Hz Ricker source near the top,
256 x 256 receivers, 1000 time steps.  One benchmark step is one whole shot
(1000 fused time-step launches plus the receiver gathers), run through the C
ABI (fd_run_shot) on device-resident inputs.  The fields (3 x 537 MB) are
larger than the 126 MB L2, so every time step streams from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own shot on its own GPU (independent
replicas, weak scaling, no data-path collective); the barrier and the max over
ranks of the timed region are the only collectives.

Reported beside the device-timed value: ``e2e`` (the same metric with the
velocity uploaded from pinned host memory and the traces read back every
step), ``roofline`` (the step kernel's algorithmic HBM bytes per launch over
its average launch time, against the measured copy bandwidth), ``clocks``
(nvidia-smi sampled during the timed region) and ``cpu_baseline`` (the FP64
oracle on the host cores, on a bounded sample of the same grid).  At N = 1 the
line also carries the single-GPU sections: batched 2D and 3D shots, serving,
the adjoint gradient, the paper's unfused routines and two-step fusion.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

BYTES_PER_UPDATE = 16          # read P, Pold, w; write Pn (FP32)
FALLBACK_HBM_GBS = 6400.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fd_step3d_512cube_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2311_05038_b300", "csrc", f)
                  for f in ("fd_kernels.cu", "fd_internal.h", "ptx.cuh", "stencil.cuh")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--grid", "--n", dest="n", type=int, default=512, help="cube side")
    ap.add_argument("--time-steps", "--nt", dest="nt", type=int, default=1000, help="time steps per shot")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-unfused", action="store_true")
    ap.add_argument("--skip-fused", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--adjoint-shots", type=int, default=8, help="adjoint workload: shots per gradient")
    ap.add_argument("--adjoint-lanes", type=int, default=4, help="adjoint workload: concurrent shot streams")
    ap.add_argument("--serve-shots", type=int, default=500, help="serving workload: requests in the stream")
    ap.add_argument("--workload", default="roofline3d", choices=["roofline3d", "batched", "batched3d", "serving"])
    ap.add_argument("--shots", type=int, default=64, help="batched workload: number of 2D shots")
    ap.add_argument("--batch-nt", type=int, default=2000, help="batched workload: steps per shot")
    ap.add_argument("--batch-tile", type=int, default=-1,
                    help="batched workload: fd_batch_tuning.tile (0-2 persistent, 3-7 one launch per "
                         "step); -1 autotunes")
    ap.add_argument("--group-mb", type=int, default=96, help="batched workload: group budget with --batch-tile")
    return ap.parse_args()


# ------------------------------------------------------------------------ helpers

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(n):
    """DRAM bytes per step-kernel launch from the committed ncu summary, scaled to n^3,
    or None if the summary is missing or the kernel source changed since."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_digest():
            return None
        per_point = float(kv["dram_bytes_per_launch"]) / float(kv["points_per_launch"])
        return per_point * n ** 3
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling for the duration of a with-block."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id, enabled=True):
        self.gpu_id = gpu_id
        self.enabled = enabled
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                time.sleep(0.3)
            except Exception:
                self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        loaded = [s for s in sm if smax and s > 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(dist, x: float, device="cpu") -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, elapsed_max: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / elapsed_max


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "b300" else "gloo")
        return dist, rank, local, world
    return None, 0, 0, 1


# ------------------------------------------------------------------------ oracle

def oracle_sample(shot, budget_s=15.0, max_steps=50):
    """Time the FP64 oracle on the benchmark grid for a bounded number of steps."""
    from oracle import oracle
    oracle.build()
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    P, Pold, _ = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                            src=shot.src, wavelet=shot.wavelet, receivers=None, nsteps=1)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width, src=shot.src,
               wavelet=shot.wavelet, receivers=shot.receivers, P=P, Pold=Pold, n0=1, nsteps=steps)
    el = time.perf_counter() - t0
    return steps * shot.npoints / el / 1e9, threads, steps, el


def run_reference(args, dist, rank, world):
    """The reference arm: the FP64 oracle on the host cores, same grid and metric."""
    if rank != 0:
        return
    shot = wl.roofline_3d(n=args.n, nt=args.nt)
    from oracle import oracle
    oracle.build()
    threads = oracle.max_threads()
    # size one benchmark step from a one-time-step probe (about 8 s of CPU work)
    t0 = time.perf_counter()
    P, Pold, _ = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                            src=shot.src, wavelet=shot.wavelet, nsteps=1)
    probe = time.perf_counter() - t0
    per_step = int(max(1, min(args.nt, 8.0 / max(probe, 1e-3))))
    n0 = 1

    def one():
        nonlocal P, Pold, n0
        P, Pold, _ = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                                src=shot.src, wavelet=shot.wavelet, receivers=shot.receivers,
                                P=P, Pold=Pold, n0=n0, nsteps=per_step)
        n0 += per_step

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = args.steps * per_step * shot.npoints / el / 1e9
    sample = (f"{args.n}^3 layered grid, {per_step} of {args.nt} time steps per benchmark step, "
              f"FP64 oracle (plain C loop, OpenMP over z)")
    line = {
        "impl": "reference", "metric": "Gpt-updates/s", "value": value, "unit": "Gupd/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": shot.name, "grid": list(shot.shape), "time_steps_per_bench_step": per_step,
                   "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "Gupd/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gupd/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ batched 2D

def measure_batched(nshots=64, nt=2000, repeats=1, tile=-1, group_mb=96):
    """The batched 2D workload served three ways on this GPU: one shot at a time
    (fd_run_shot per shot, back to back on one stream), one shot at a time on
    each of 8 streams at once, and all shots in one persistent batch
    (autotuned).  Returns a summary dict; results are compared bitwise."""
    import torch
    from paper_2311_05038_b300 import fd
    shapes = wl.batched_2d_shapes(nshots)
    shots = [wl.batched_2d_shot(i, s, nt) for i, s in enumerate(shapes)]
    updates = sum(s.npoints for s in shots) * nt
    models = [fd.Model.from_shot(s) for s in shots]

    def plain():
        for m in models:
            m.run_shot(nt)
        for m in models:
            fd.fd_synchronize(m.handle)

    def timed(fn):
        fn()                                  # warm-up pass
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(repeats):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / repeats

    launches0 = fd.fd_kernel_launch_count()
    t_plain = timed(plain)
    plain_launches = (fd.fd_kernel_launch_count() - launches0) // (repeats + 1)
    ref = [m.traces(nt).copy() for m in models]
    ref_p = [m.wavefield() for m in models[:8]]
    # one shot at a time per stream, on `nstreams` streams at once (fd_run_shot per
    # shot; shot i on stream i mod nstreams)
    nstreams = 8
    handles = [fd.fd_stream_create(0)[0] for _ in range(nstreams)]
    smodels = [fd.Model.from_shot(s, stream=handles[i % nstreams]) for i, s in enumerate(shots)]

    def streams():
        for m in smodels:
            m.run_shot(nt)
        for m in smodels:
            fd.fd_synchronize(m.handle)

    t_streams = timed(streams)
    same_streams = all(np.array_equal(m.traces(nt), r) for m, r in zip(smodels, ref))
    for m in smodels:
        m.close()
    for h in handles:
        fd.fd_stream_destroy(h)
    batch = fd.Batch(models)
    if tile >= 0:
        batch.set_tuning(tile=tile, steps_per_launch=nt, ctas_per_sm=0, group_mb=group_mb)
        tuning = batch.tuning()
    else:
        tuning = batch.autotune(trial_steps=20)
    launches0 = fd.fd_kernel_launch_count()
    t_batch = timed(lambda: batch.run_shots([nt] * nshots))
    batch_launches = (fd.fd_kernel_launch_count() - launches0) // (repeats + 1)
    same = all(np.array_equal(m.traces(nt), r) for m, r in zip(models, ref)) and \
        all(np.array_equal(m.wavefield(), p) for m, p in zip(models[:8], ref_p))
    batch.close()
    for m in models:
        m.close()
    peak, _ = measured_hbm_peak()
    return {
        "workload": f"{nshots} 2D shots {min(shapes)}..{max(shapes)} (nz, nx), GRF velocity, sponge 20, {nt} steps",
        "updates": updates,
        "plain": {"s": t_plain, "shots_per_s": nshots / t_plain, "gupd": updates / t_plain / 1e9,
                  "launches": int(plain_launches)},
        "plain_streams": {"streams": nstreams, "s": t_streams, "shots_per_s": nshots / t_streams,
                          "gupd": updates / t_streams / 1e9, "results_identical": bool(same_streams)},
        "batched": {"s": t_batch, "shots_per_s": nshots / t_batch, "gupd": updates / t_batch / 1e9,
                    "frac": 16 * updates / t_batch / 1e9 / peak, "launches": int(batch_launches),
                    "tuning": tuning},
        "speedup": t_plain / t_batch,
        "speedup_vs_streams": t_streams / t_batch,
        "results_identical": bool(same),
    }


def measure_batched_3d(nshots=24, nt=300, seed=6):
    """Uneven 3D shots (cubes 128..256 of the serving mix, layered + random velocity,
    sponge 20) served three ways: one shot at a time on one stream, one at a time
    on each of 8 streams at once, and all in one batch (one launch per time step
    over every model).  Results are compared bitwise."""
    import torch
    from paper_2311_05038_b300 import fd
    shots = wl.batched_3d_shots(nshots, nt, seed)
    sizes = np.array([s.shape[0] for s in shots])
    updates = sum(s.npoints for s in shots) * nt

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    models = [fd.Model.from_shot(s) for s in shots]

    def plain():
        for m in models:
            m.run_shot(nt)
        for m in models:
            fd.fd_synchronize(m.handle)

    t_plain = timed(plain)
    ref = [m.traces(nt).copy() for m in models]
    handles = [fd.fd_stream_create(0)[0] for _ in range(8)]
    smodels = [fd.Model.from_shot(s, stream=handles[i % 8]) for i, s in enumerate(shots)]

    def streams():
        for m in smodels:
            m.run_shot(nt)
        for m in smodels:
            fd.fd_synchronize(m.handle)

    t_streams = timed(streams)
    same_streams = all(np.array_equal(m.traces(nt), r) for m, r in zip(smodels, ref))
    for m in smodels:
        m.close()
    for h in handles:
        fd.fd_stream_destroy(h)
    batch = fd.Batch(models)
    t_batch = timed(lambda: batch.run_shots([nt] * nshots))
    same = all(np.array_equal(m.traces(nt), r) for m, r in zip(models, ref))
    batch.close()
    for m in models:
        m.close()
    peak, _ = measured_hbm_peak()
    arm = lambda t: {"s": t, "shots_per_s": nshots / t, "gupd": updates / t / 1e9}
    return {"workload": f"{nshots} 3D shots, cubes {int(sizes.min())}..{int(sizes.max())}, {nt} steps, sponge 20",
            "plain": arm(t_plain), "plain_streams": dict(arm(t_streams), streams=8,
                                                         results_identical=bool(same_streams)),
            "batched": dict(arm(t_batch), frac=16 * updates / t_batch / 1e9 / peak), "speedup": t_plain / t_batch, "speedup_vs_streams": t_streams / t_batch,
            "results_identical": bool(same)}


def measure_2d_large(n=8192, nt=200):
    """One large 2D shot (n x n, GRF-free layered-constant velocity 2000 m/s, sponge
    20): device Gupd/s of fd_step, 16 algorithmic bytes per update."""
    import torch
    from paper_2311_05038_b300 import fd
    vel = np.full((n, n), 2000.0, np.float32)
    dt = wl.courant_dt(10.0, 2000.0)
    rec = np.array([(ix, 0, 32) for ix in range(0, n, 4)], np.int32)
    shot = wl.Shot(2, (n, n), 10.0, dt, nt, vel, (n // 2, 0, n // 2), wl.ricker(nt, dt, 15.0), rec, sponge_width=20)
    stream = torch.cuda.Stream()
    with fd.Model.from_shot(shot, stream=stream) as m:
        m.run_shot(20)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.run_shot(nt)
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    peak, _ = measured_hbm_peak()
    gupd = n * n * nt / t / 1e9
    return {"workload": f"2D {n}x{n}, {nt} steps, sponge 20", "gupd": gupd, "frac": 16 * gupd / peak}


# ------------------------------------------------------------------------ serving 3D

def measure_serving(nshots=500, closed_shots=100, max_active=4, load=0.8, budget_gb=150):
    """The serving workload: a Poisson stream of 3D shots (cubes 128..384, 200..2000
    steps) served by continuous batching and one at a time.  Open loop: the whole
    stream, arrivals at `load` times the one-at-a-time service rate (calibrated
    here), reporting p50/p99 latency.  Closed loop: the first `closed_shots`
    requests queued at t = 0, reporting shots/s.  Traces are compared bitwise
    between the modes."""
    import torch
    from paper_2311_05038_b300 import fd, serving
    sizes = list(range(128, 385, 32))
    cache = {}
    for n in sizes:
        for k in range(2):
            cache[(n, k)] = torch.from_numpy(wl.serving_3d_velocity(n, 4000 + 10 * n + k)).pin_memory()
    per_step = {}
    for n in sizes:
        shot = wl.serving_3d_shot(0, n, 100, vel=cache[(n, 0)].numpy())
        with fd.Model.from_shot(shot) as m:
            m.run_shot(20)
            fd.fd_synchronize(m.handle)
            t0 = time.perf_counter()
            m.run_shot(100)
            fd.fd_synchronize(m.handle)
            per_step[n] = (time.perf_counter() - t0) / 100
    base = wl.serving_3d_stream(nshots, seed=4, rate=1.0)
    mean_service = float(np.mean([nt * per_step[n] for _, n, nt in base]))
    rate = load / mean_service
    stream = wl.serving_3d_stream(nshots, seed=4, rate=rate)
    reqs = []
    for i, (arr, n, nt) in enumerate(stream):
        vel = cache[(n, i % 2)]
        reqs.append(serving.Request(i, arr, wl.serving_3d_shot(i, n, nt, vel=vel.numpy()), vel))
    closed_shots = min(closed_shots, nshots)
    out = {"workload": f"{nshots} 3D shots (open loop; closed loop: the first {closed_shots}), cubes 128..384, "
                       f"200..2000 steps, Poisson arrivals at {load} x the one-at-a-time service rate",
           "rate_per_s": rate, "mean_service_s_one_at_a_time": mean_service, "budget_gb": budget_gb,
           "max_active": max_active}
    traces = {}
    for mode, ma in (("continuous", max_active), ("one_at_a_time", 1)):
        srv = serving.Server(max_active=ma, budget_bytes=int(budget_gb * 1e9), chunk=100, depth=2, max_nt=2000)
        srv.serve(reqs[:4], realtime=False)                      # warm the pool
        t0 = time.perf_counter()
        res = srv.serve(reqs, realtime=True)
        open_loop = serving.summarize(res, time.perf_counter() - t0)
        t0 = time.perf_counter()
        res_c = srv.serve(reqs[:closed_shots], realtime=False)
        closed = serving.summarize(res_c, time.perf_counter() - t0)
        out[mode] = {"policy": srv.policy, "open_loop": open_loop, "closed_loop": closed,
                     "peak_hbm_gb": srv.pool.peak / 1e9}
        traces[mode] = [r.traces for r in res]
        srv.close()
    out["results_identical"] = all(np.array_equal(a, b) for a, b in zip(traces["continuous"],
                                                                       traces["one_at_a_time"]))
    out["closed_loop_speedup"] = (out["continuous"]["closed_loop"]["shots_per_s"] /
                                  out["one_at_a_time"]["closed_loop"]["shots_per_s"])
    return out


# ------------------------------------------------------------------------ adjoint 3D

def measure_adjoint(n=256, nt=1500, nshots=8, checkpoint_every=50, lanes=4):
    """Gradient of the trace misfit w.r.t. squared slowness for the adjoint
    workload (observed data from the +5 % anomaly model): time per gradient
    over all shots, the forward share, and the device memory it held.  The
    headline runs the shots on `lanes` concurrent streams (adjoint.ShotLanes);
    the same gradient one shot at a time on one stream, and keeping every L'P^n
    instead of checkpoints, are reported beside it."""
    import torch
    from paper_2311_05038_b300 import adjoint, fd
    shots, v_true = wl.adjoint_3d(n, nt, nshots)
    vmax = 4000.0 * 1.05
    observed = []
    for s in shots:
        s2 = wl.Shot(3, s.shape, s.h, s.dt, nt, v_true, s.src, s.wavelet, s.receivers, sponge_width=s.sponge_width)
        with fd.Model.from_shot(s2) as m:
            fd.fd_set_sponge_vmax(m.handle, vmax)
            m.run_shot(nt)
            observed.append(torch.from_numpy(m.traces(nt)).cuda())
    m0 = torch.from_numpy((1.0 / shots[0].vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    geos = [adjoint.Geometry.from_shot(s, checkpoint_every=checkpoint_every, sponge_vmax=vmax) for s in shots]
    # untimed warm-up gradients on a small cut of the workload: load the device code
    # of every op on both paths (casts, FP64 reduction, autograd) before timing
    wshots, _ = wl.adjoint_3d(48, 40, 2)
    wgeos = [adjoint.Geometry.from_shot(w, checkpoint_every=10, sponge_vmax=vmax) for w in wshots]
    wm = torch.from_numpy((1.0 / wshots[0].vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    wobs = [torch.zeros((40, len(wshots[0].receivers)), device="cuda")] * 2
    adjoint.misfit_and_gradient(wm, wgeos[0], wobs[0])
    wl_lanes = adjoint.ShotLanes(wgeos, lanes=2)
    wl_lanes.run(wm, wobs)
    wl_lanes.close()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    t0 = time.perf_counter()
    eng = adjoint.ShotLanes(geos, lanes=lanes)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    J, grad = eng.run(m0, observed)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    t0 = time.perf_counter()
    Jf, _ = eng.run(m0, observed, backward=False)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    peak = torch.cuda.max_memory_allocated() - base
    eng.close()
    del eng
    torch.cuda.empty_cache()
    # one shot at a time on one stream (Propagate per shot)
    t0 = time.perf_counter()
    grad_1 = torch.zeros_like(m0)
    for g, dobs in zip(geos, observed):
        grad_1 += adjoint.misfit_and_gradient(m0, g, dobs)[1]
    torch.cuda.synchronize()
    el_1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    for g in geos:
        with torch.no_grad():
            adjoint.Propagate.apply(m0, g)
    torch.cuda.synchronize()
    fwd_1 = time.perf_counter() - t0
    rel_1 = float((grad_1 - grad).double().norm() / grad_1.double().norm())
    # the same gradient keeping every L'P^n instead of checkpoints (nt fields per shot)
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    t0 = time.perf_counter()
    grad_s = torch.zeros_like(m0)
    for s, dobs in zip(shots, observed):
        geo = adjoint.Geometry.from_shot(s, sponge_vmax=vmax, store_all=True)
        grad_s += adjoint.misfit_and_gradient(m0, geo, dobs)[1]
    torch.cuda.synchronize()
    el_s = time.perf_counter() - t0
    peak_s = torch.cuda.max_memory_allocated() - base
    same = bool(torch.equal(grad_1, grad_s))
    del grad_s, grad_1
    torch.cuda.empty_cache()
    return {"workload": f"{nshots} shots, {n}^3, {nt} steps, checkpoints every {checkpoint_every}",
            "lanes": lanes, "s_per_gradient": el, "forward_s": fwd, "gradient_over_forward": el / fwd,
            "misfit": J, "setup_s": setup, "peak_torch_memory_gb": peak / 1e9,
            "gupd_forward": nshots * nt * n ** 3 / fwd / 1e9,
            "gupd_forward_equivalent": nshots * nt * n ** 3 / el / 1e9, "grad_norm": float(grad.norm()),
            "one_stream": {"s_per_gradient": el_1, "forward_s": fwd_1, "gupd_forward": nshots * nt * n ** 3 / fwd_1 / 1e9,
                           "gradient_rel_l2_vs_lanes": rel_1},
            "store_all": {"s_per_gradient": el_s, "gradient_over_forward": el_s / fwd_1,
                          "peak_torch_memory_gb": peak_s / 1e9, "gradient_identical_to_one_stream": same}}


# ------------------------------------------------------------------------ fused pairs 3D

def measure_time_fusion(shot, model, stream, traces, shots=3):
    """The benchmark shot with two time steps per launch (fd_set_time_fusion): Gupd/s
    over `shots` whole shots (one warm-up shot first), 10 algorithmic bytes per
    update, and the traces compared bitwise with the single-step run's."""
    import torch
    from paper_2311_05038_b300 import fd
    ref = traces.clone()
    m2 = fd.Model.from_shot(shot, stream=stream)
    m2.set_time_fusion(2)
    m2.run_shot(shot.nt, traces)
    torch.cuda.synchronize()
    same = bool(torch.equal(traces, ref))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = fd.fd_kernel_launch_count()
    e0.record(stream)
    for _ in range(shots):
        m2.run_shot(shot.nt, traces)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = fd.fd_kernel_launch_count() - l0
    t = e0.elapsed_time(e1) / 1e3
    m2.close()
    peak, _ = measured_hbm_peak()
    npts = shot.npoints
    pair_s = t / (shots * shot.nt / 2)
    return {"gupd": shots * shot.nt * npts / t / 1e9, "ms_per_shot": t / shots * 1e3,
            "avg_pair_launch_us": pair_s * 1e6, "launches_per_shot": launches / shots,
            "bytes_per_update": 10, "achieved_GBs": 20 * npts / pair_s / 1e9,
            "frac_algorithmic": 20 * npts / pair_s / 1e9 / peak, "traces_identical_to_single_steps": same}


# ------------------------------------------------------------------------ unfused 3D

def measure_unfused(shot, model, stream, reps=20):
    """Per-routine times of the paper's unfused sequence on the benchmark grid,
    each against its own algorithmic bytes, and the whole unfused step."""
    import torch
    from paper_2311_05038_b300 import fd
    npts = shot.npoints
    routines = [("fd_pzz", fd.FD_ROUTINE_PZZ, 8), ("fd_pxx", fd.FD_ROUTINE_PXX, 8), ("fd_pyy", fd.FD_ROUTINE_PYY, 8),
                ("fd_time", fd.FD_ROUTINE_TIME, 28)]
    peak, _ = measured_hbm_peak()
    out = {}
    for name, r, bpp in routines:
        fd.fd_routine(model.handle, r)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fd.fd_routine(model.handle, r)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"us": t * 1e6, "bytes_per_update": bpp, "GBs": bpp * npts / t / 1e9,
                     "frac": bpp * npts / t / 1e9 / peak}
    fd.fd_reset(model.handle)
    fd.fd_step_unfused(model.handle, 2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fd.fd_step_unfused(model.handle, reps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    return {"routines": out, "step_us": t * 1e6, "gupd": npts / t / 1e9, "bytes_per_update": 52,
            "note": "the paper's add_source, fd_pzz, fd_pxx, fd_pyy, fd_time, swap as separate kernels"}


# ------------------------------------------------------------------------ main arm

def run_b300(args, dist, rank, local, world):
    import torch
    torch.cuda.set_device(local)
    from paper_2311_05038_b300 import fd

    shot = wl.roofline_3d(n=args.n, nt=args.nt)
    npts = shot.npoints
    stream = torch.cuda.Stream()
    model = fd.Model.from_shot(shot, stream=stream)
    nrec = len(shot.receivers)
    traces = torch.empty((shot.nt, nrec), device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident timed region
    for _ in range(args.warmup):
        model.run_shot(shot.nt, traces)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else local
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    launches0 = fd.fd_kernel_launch_count()
    with ClockSampler(gpu_id, enabled=not args.no_clocks) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            model.run_shot(shot.nt, traces)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = fd.fd_kernel_launch_count() - launches0
    fd.fd_synchronize(model.handle)
    barrier()
    elapsed = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, "cuda")
    value = replica_throughput(args.steps * shot.nt * npts, world, elapsed) / 1e9
    step_launches = args.steps * shot.nt
    avg_launch_s = ev0.elapsed_time(ev1) / 1e3 / step_launches
    achieved = BYTES_PER_UPDATE * npts / avg_launch_s / 1e9
    peak, peak_kind = measured_hbm_peak()

    fused = None
    # the single-GPU sections run at N = 1 only: under torchrun they would hold
    # every rank's GPU while rank 0 alone works
    extras = rank == 0 and world == 1
    if extras and not args.skip_fused:
        fused = measure_time_fusion(shot, model, stream, traces, args.steps)

    unfused = None
    if extras and not args.skip_unfused:
        unfused = measure_unfused(shot, model, stream)

    # ---- end to end: velocity up from pinned host memory, traces back, every step.
    # Two models on two streams take alternate shots, so one shot's upload and
    # the previous shot's trace download run on the copy engines while the
    # other model computes; every copy is inside the timed region.
    e2e = None
    if not args.skip_e2e:
        v_pinned = torch.from_numpy(shot.vel.ravel()).pin_memory()
        tr_pinned = [torch.empty((shot.nt, nrec), dtype=torch.float32).pin_memory() for _ in range(2)]
        rec = shot.receivers
        stream2 = torch.cuda.Stream()
        models = [model, fd.Model.from_shot(shot, stream=stream2)]

        def e2e_step(k):
            m = models[k % 2]
            fd.fd_set_velocity_ptr(m.handle, v_pinned.data_ptr())
            m.set_source(shot.src, shot.wavelet)
            m.set_receivers(rec)
            m.run_shot(shot.nt)
            fd.fd_gather_traces_async_ptr(m.handle, tr_pinned[k % 2].data_ptr(), tr_pinned[k % 2].numel())

        for k in range(2):
            e2e_step(k)
        for m in models:
            fd.fd_synchronize(m.handle)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(k)
        for m in models:
            fd.fd_synchronize(m.handle)
        el = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
        models[1].close()
        h2d = shot.vel.nbytes + shot.wavelet.nbytes + rec.nbytes
        d2h = shot.nt * nrec * 4
        e2e = {"value": world * args.steps * shot.nt * npts / el / 1e9, "unit": "Gupd/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "overlap": "two models on two streams alternate shots; uploads and downloads overlap compute"}
    model.close()

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        del traces
        torch.cuda.empty_cache()
        v, threads, steps, el = oracle_sample(shot)
        cpu = {"value": v, "unit": "Gupd/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.n}^3 layered grid with sponge, source and receivers, {steps} of "
                         f"{args.nt} time steps, FP64 oracle, {el:.1f} s"}

    batched = batched3 = None
    if extras and not args.skip_batched:
        torch.cuda.empty_cache()
        batched = measure_batched(args.shots, args.batch_nt)
        batched3 = measure_batched_3d()
        batched["single_shot_2d_large"] = measure_2d_large()
    adj = None
    if extras and not args.skip_adjoint:
        torch.cuda.empty_cache()
        adj = measure_adjoint(nshots=args.adjoint_shots, lanes=args.adjoint_lanes)
    served = None
    if extras and not args.skip_serving:
        torch.cuda.empty_cache()
        served = measure_serving(args.serve_shots)

    if rank == 0:
        traffic = recorded_traffic(args.n)
        line = {
            "metric": "Gpt-updates/s", "value": value, "unit": "Gupd/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": shot.name, "grid": list(shot.shape), "time_steps_per_bench_step": shot.nt,
                       "receivers": nrec, "sponge": shot.sponge_width,
                       "l2": "fields (3 x %.0f MB) larger than L2; no flush needed" % (npts * 4 / 1e6),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": traffic, "kernel": "fdk::step3d_kernel",
                         "algorithmic_bytes_per_launch": BYTES_PER_UPDATE * npts,
                         "avg_launch_us": avg_launch_s * 1e6},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks.summary(),
            "gpu_launches": int(launches),
            "batched_2d": batched,
            "batched_3d": batched3,
            "serving_3d": served,
            "adjoint_3d": adj,
            "unfused_3d": unfused,
            "time_fusion_3d": fused,
        }
        print(json.dumps(line), flush=True)


def run_batched_line(args, rank):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if rank != 0:
        return
    r = measure_batched(args.shots, args.batch_nt, repeats=max(1, args.steps), tile=args.batch_tile,
                        group_mb=args.group_mb)
    line = {"metric": "shots/s (batched 2D)", "value": r["batched"]["shots_per_s"], "unit": "shots/s",
            "n_gpus": 1, "steps": max(1, args.steps), "warmup": 1, "ms_per_step": r["batched"]["s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r}
    print(json.dumps(line), flush=True)


def run_batched3d_line(args, rank):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if rank != 0:
        return
    r = measure_batched_3d()
    line = {"metric": "shots/s (batched 3D)", "value": r["batched"]["shots_per_s"], "unit": "shots/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": r["batched"]["s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r}
    print(json.dumps(line), flush=True)


def run_serving_line(args, rank):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if rank != 0:
        return
    r = measure_serving(args.serve_shots)
    c = r["continuous"]
    line = {"metric": "shots/s (served 3D, continuous batching)", "value": c["closed_loop"]["shots_per_s"],
            "unit": "shots/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": c["closed_loop"]["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": {"workload": r["workload"]},
            "p50_s": c["open_loop"]["p50_s"], "p99_s": c["open_loop"]["p99_s"], "detail": r}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist, rank, local, world = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, dist, rank, world)
        elif args.workload == "batched":
            run_batched_line(args, rank)
        elif args.workload == "batched3d":
            run_batched3d_line(args, rank)
        elif args.workload == "serving":
            run_serving_line(args, rank)
        else:
            run_b300(args, dist, rank, local, world)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
