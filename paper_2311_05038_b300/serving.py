"""Continuous-batching server for 3D shots on one GPU.

A request is one shot (grid, velocity, source, receivers, step count) with an
arrival time.  The server keeps a set of active shots whose wavefields stay
resident on the device; each advances on a CUDA stream of its own, in chunks of
time steps (``fd_step``), with up to ``depth`` chunks queued, so the kernels of
several shots run on the GPU at the same time.  When a shot's last chunk
completes, its traces are read back and its model returns to a pool.

Admission.  Requests that arrive while others run wait in arrival order and are
admitted as soon as a slot is free and their device memory fits the HBM budget.
A request that does not fit yet lets later requests that do fit pass it, at
most ``max_bypass`` times; after that nothing passes it until it is admitted,
so no request starves.

Priorities.  Overlap alone shares the GPU evenly between the active shots,
which stretches the longest shots and so the latency tail.  Each active shot's
stream therefore carries a priority, by default from an earliest-deadline
ranking (a shot is due a fixed multiple of its stand-alone time after it
arrives), so the block scheduler gives the most urgent shot the SMs it can use
and fills the rest (tail waves, gaps between launches, small grids) with the
others' blocks.  A shot changes priority by moving to another stream of its
own (``fd_set_stream``, which keeps its work in order).

Models are pooled per grid and reused for later requests of the same grid
instead of being freed: ``cudaFree`` synchronises the whole device and would
stall every running shot.  An idle pooled model of another grid is released
only when a new grid does not otherwise fit the budget.

The propagation itself is libfd's (the same fused step kernels as ``fd_step``),
so every shot gives bitwise the same traces alone and in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import fd


# ------------------------------------------------------------------ requests

@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of serving
    shot: object                # a workloads.Shot (3D)
    vel_pinned: object = None   # optional pinned torch tensor holding shot.vel (fast upload)


@dataclass
class Result:
    rid: int
    traces: np.ndarray
    arrival: float
    admitted: float
    done: float
    updates: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def model_key(shot, max_nt: int):
    """Requests with equal keys can reuse one pooled model."""
    return (tuple(shot.shape), float(shot.h), float(shot.dt), int(shot.sponge_width), float(shot.sponge_R),
            int(len(shot.receivers)), int(max_nt))


def footprint_bytes(shot, max_nt: int) -> int:
    """Device memory one pooled model holds: P, Pold, w and the velocity staging
    copy (row pitch rounded to 32 floats) plus a trace buffer of max_nt rows."""
    nz, ny, nx = shot.shape
    px = (nx + 31) // 32 * 32
    return 4 * 4 * nz * ny * px + 4 * max_nt * len(shot.receivers) + 4 * max_nt


# ------------------------------------------------------------------ pool accounting

class ModelPool:
    """Pooled models per key under a byte budget (no CUDA here: ``create`` and
    ``destroy`` are supplied by the caller, which keeps the policy testable)."""

    def __init__(self, budget_bytes: int, create, destroy):
        self.budget = int(budget_bytes)
        self.create = create
        self.destroy = destroy
        self.idle = collections.OrderedDict()   # key -> list of idle models (LRU order of keys)
        self.used = 0
        self.peak = 0
        self.sizes = {}                          # id(model) -> bytes

    def acquire(self, key, nbytes: int):
        """An idle model for key, a new one if the budget allows (releasing idle
        models of other keys if that makes room), else None."""
        lst = self.idle.get(key)
        if lst:
            m = lst.pop()
            if not lst:
                del self.idle[key]
            return m
        if nbytes > self.budget:
            raise ValueError(f"one model needs {nbytes} B, more than the budget {self.budget} B")
        while self.used + nbytes > self.budget:
            victim = next((k for k in self.idle if k != key and self.idle[k]), None)
            if victim is None:
                return None
            vm = self.idle[victim].pop()
            if not self.idle[victim]:
                del self.idle[victim]
            self.used -= self.sizes.pop(id(vm))
            self.destroy(vm)
        m = self.create(key)
        self.sizes[id(m)] = nbytes
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        return m

    def release(self, key, m):
        self.idle.setdefault(key, []).append(m)
        self.idle.move_to_end(key)

    def close(self):
        for lst in self.idle.values():
            for m in lst:
                self.used -= self.sizes.pop(id(m), 0)
                self.destroy(m)
        self.idle.clear()


def percentile(values, q):
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sequence."""
    v = sorted(values)
    if not v:
        return float("nan")
    k = max(0, min(len(v) - 1, int(np.ceil(q / 100.0 * len(v))) - 1))
    return float(v[k])


# ------------------------------------------------------------------ scheduling policy

def admit_in_order(waiting, free_slots, bypassed, max_bypass, try_admit):
    """Admit from ``waiting`` (a list in arrival order, modified in place) into at
    most ``free_slots`` slots.  ``try_admit(request)`` returns the admitted entry or
    None when the request does not fit yet; a request that does not fit lets later
    ones pass it until ``max_bypass`` of them have (``bypassed`` counts them for the
    current head and is returned updated), after which nothing passes it.
    Returns (admitted entries, bypassed)."""
    out = []
    i = 0
    while i < len(waiting) and len(out) < free_slots:
        if i > 0 and bypassed >= max_bypass:
            break
        a = try_admit(waiting[i])
        if a is None:
            i += 1
            continue
        del waiting[i]
        bypassed = bypassed + 1 if i > 0 else 0
        out.append(a)
    return out, bypassed


def rank_active(active, policy, slack=2.0, rate=300e9):
    """Active shots in priority order.  Each entry needs ``arrival``, ``rid``,
    ``npoints``, ``nt`` and ``work_left``.  "age": oldest first; "oldest+srpt":
    the oldest, then least remaining work; "deadline": earliest arrival + slack x
    stand-alone time (npoints x nt / rate)."""
    if policy == "age":
        return sorted(active, key=lambda a: (a.arrival, a.rid))
    if policy == "oldest+srpt":
        oldest = min(active, key=lambda a: (a.arrival, a.rid))
        rest = sorted((a for a in active if a is not oldest), key=lambda a: (a.work_left, a.rid))
        return [oldest] + rest
    if policy == "deadline":
        return sorted(active, key=lambda a: (a.arrival + slack * a.npoints * a.nt / rate, a.rid))
    raise ValueError(f"unknown policy {policy!r}")


# ------------------------------------------------------------------ server

@dataclass
class _Active:
    req: Request
    model: object
    key: tuple
    admitted: float
    remaining: int              # steps not yet issued
    inflight: collections.deque = field(default_factory=collections.deque)   # (event, steps)

    @property
    def work_left(self) -> int:
        """Grid-point updates not yet completed."""
        return (self.remaining + sum(k for _, k in self.inflight)) * int(self.req.shot.npoints)

    @property
    def arrival(self):
        return self.req.arrival

    @property
    def rid(self):
        return self.req.rid

    @property
    def npoints(self):
        return int(self.req.shot.npoints)

    @property
    def nt(self):
        return int(self.req.shot.nt)


class Server:
    """Continuous-batching server over libfd models on the current CUDA device.

    max_active  shots whose work may be on the GPU at once (1 = one at a time)
    budget_bytes  HBM the pooled models may hold
    chunk       time steps per fd_step call; depth: chunks queued per shot
    max_nt      largest step count a request may ask for (trace buffers are
                sized for it once per pooled model)
    policy      how active shots are ranked onto stream priorities: "age"
                (oldest first), "oldest+srpt" (the oldest, then shortest
                remaining work), "deadline" (earliest arrival + slack x the
                shot's work at ``rate_gupd``), or "none" (all at the default
                priority).  Default "deadline" when more than one shot may be
                active, else "none".
    max_bypass  how many later requests may be admitted ahead of a waiting
                request that does not fit yet
    """

    def __init__(self, max_active=4, budget_bytes=150 * 10**9, chunk=100, depth=2, max_nt=2000,
                 policy=None, max_bypass=8, slack=2.0, rate_gupd=300.0):
        import torch
        self.torch = torch
        self.max_active = int(max_active)
        self.chunk = int(chunk)
        self.depth = int(depth)
        self.max_nt = int(max_nt)
        if policy is None:
            policy = "deadline" if self.max_active > 1 else "none"
        if policy not in ("age", "oldest+srpt", "deadline", "none"):
            raise ValueError(f"unknown policy {policy!r}")
        self.policy = policy
        self.slack = float(slack)
        self.rate = float(rate_gupd) * 1e9
        self.max_bypass = int(max_bypass)
        self.greatest = None             # the device's highest stream priority, once known
        self.pool = ModelPool(budget_bytes, self._create, self._destroy)

    # -- streams: each pooled model owns one library stream per priority it has used
    def _stream(self, m, prio):
        if prio not in m.streams:
            handle, greatest = fd.fd_stream_create(prio)
            self.greatest = greatest
            m.streams[prio] = (handle, self.torch.cuda.ExternalStream(handle))
        return m.streams[prio]

    def _set_priority(self, m, prio):
        if m.prio != prio:
            handle, _ = self._stream(m, prio)
            fd.fd_set_stream(m.handle, handle)
            m.prio = prio

    # -- pool callbacks
    def _create(self, key):
        shape, h, dt, W, R, nrec, max_nt = key
        vel = np.full(shape, 1500.0, np.float32)
        streams = {}
        handle, greatest = fd.fd_stream_create(0)
        self.greatest = greatest
        streams[0] = (handle, self.torch.cuda.ExternalStream(handle))
        m = fd.Model(3, shape, h, dt, vel, W, R, stream=handle)
        m.streams = streams
        m.prio = 0
        # reserve the per-request buffers once: receivers, source signature, traces
        m.set_receivers(np.zeros((nrec, 3), np.int32))
        m.set_source((0, 0, 0), np.zeros(max_nt, np.float32))
        fd.fd_set_trace_buffer(m.handle, None, max_nt)
        return m

    def _destroy(self, m):
        m.close()                       # waits for the model's current stream, which is ordered last
        for handle, _ in m.streams.values():
            fd.fd_stream_destroy(handle)
        m.streams = {}

    # -- one request
    def _admit(self, req: Request, now: float):
        shot = req.shot
        if shot.nt > self.max_nt:
            raise ValueError(f"request {req.rid}: {shot.nt} steps exceed max_nt {self.max_nt}")
        key = model_key(shot, self.max_nt)
        m = self.pool.acquire(key, footprint_bytes(shot, self.max_nt))
        if m is None:
            return None
        if req.vel_pinned is not None:
            fd.fd_set_velocity_ptr(m.handle, req.vel_pinned.data_ptr())
        else:
            fd.fd_set_velocity(m.handle, shot.vel, shot.npoints)
        m.set_source(shot.src, shot.wavelet)
        m.set_receivers(shot.receivers)
        fd.fd_reset(m.handle)
        fd.fd_set_trace_buffer(m.handle, None, shot.nt)
        return _Active(req, m, key, now, shot.nt)

    def _rank(self, active):
        """Active shots in priority order under the server's policy."""
        return rank_active(active, self.policy, self.slack, self.rate)

    def _reprioritise(self, active):
        """Priorities from the device's greatest down to 0 (the default) in rank
        order; the shots beyond the available levels stay at 0."""
        if self.policy == "none" or not active:
            return
        top = self.greatest if self.greatest is not None else 0
        for i, a in enumerate(self._rank(active)):
            self._set_priority(a.model, min(0, top + i))

    def serve(self, requests, realtime=True):
        """Serve the requests (arrival times relative to the call); returns the
        results in request order.  With realtime=False every request is treated as
        arrived at the start (closed loop), and latencies count from there."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        waiting = []                      # arrived, not admitted, in arrival order
        bypassed = 0                      # admissions ahead of waiting[0]
        active = []
        results = {}
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            progressed = False
            admitted, bypassed = admit_in_order(waiting, self.max_active - len(active), bypassed,
                                                self.max_bypass, lambda q: self._admit(q, now))
            if admitted:
                active.extend(admitted)
                progressed = True
            if progressed:
                self._reprioritise(active)
            for a in active:
                while a.remaining > 0 and len(a.inflight) < self.depth:
                    k = min(self.chunk, a.remaining)
                    fd.fd_step(a.model.handle, k)
                    ev = torch.cuda.Event()
                    ev.record(a.model.streams[a.model.prio][1])
                    a.inflight.append((ev, k))
                    a.remaining -= k
                    progressed = True
            finished = False
            for a in list(active):
                while a.inflight and a.inflight[0][0].query():
                    a.inflight.popleft()
                    progressed = True
                if a.remaining == 0 and not a.inflight:
                    nt = a.req.shot.nt
                    tr = a.model.traces(nt)
                    done = time.perf_counter() - t0
                    arrival = a.req.arrival if realtime else 0.0
                    results[a.req.rid] = Result(a.req.rid, tr, arrival, a.admitted, done,
                                                int(a.req.shot.npoints) * nt)
                    self.pool.release(a.key, a.model)
                    active.remove(a)
                    progressed = finished = True
            if finished:
                self._reprioritise(active)
            if not progressed:
                if active:
                    time.sleep(2e-5)
                elif pending and not waiting:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 1e-3)))
        return [results[r.rid] for r in requests]

    def close(self):
        self.pool.close()


def summarize(results, wall=None):
    """shots/s, updates/s and latency percentiles of a served stream."""
    lat = [r.latency for r in results]
    span = wall if wall is not None else max(r.done for r in results) - min(r.arrival for r in results)
    ups = sum(r.updates for r in results)
    return {"shots": len(results), "makespan_s": span, "shots_per_s": len(results) / span,
            "gupd": ups / span / 1e9, "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "mean_s": float(np.mean(lat))}
