"""Continuous-batching server: results are the same alone and in the mix (needs a CUDA device)."""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def stream(n=10, seed=90):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        size = int(rng.choice([48, 64, 80, 96]))
        nt = int(rng.integers(40, 160))
        shot = wl.serving_3d_shot(i, size, nt, seed=seed, sponge_width=8)
        reqs.append((i, float(0.002 * i), shot))
    return reqs


def alone(fd, shot):
    with fd.Model.from_shot(shot) as m:
        m.run_shot(shot.nt)
        return m.traces(shot.nt)


def test_results_same_alone_and_in_the_mix(fdlib):
    from paper_2311_05038_b300 import serving
    reqs = [serving.Request(i, t, s) for i, t, s in stream()]
    srv = serving.Server(max_active=4, chunk=25, depth=2, max_nt=200)
    try:
        res = srv.serve(reqs)
    finally:
        srv.close()
    assert [r.rid for r in res] == [q.rid for q in reqs]
    for q, r in zip(reqs, res):
        np.testing.assert_array_equal(r.traces, alone(fdlib, q.shot))
        assert r.done >= r.admitted >= r.arrival - 1e-9


def test_served_shots_match_the_oracle(fdlib, oracle):
    """Two shots served in a mix of four, with stream priorities changing while
    they run, against the FP64 oracle (rel L2 <= 1e-4 on the traces)."""
    from paper_2311_05038_b300 import serving
    reqs = [serving.Request(i, 0.0, s) for i, _, s in stream(n=4, seed=92)]
    srv = serving.Server(max_active=4, chunk=20, depth=1, max_nt=200)
    try:
        res = srv.serve(reqs, realtime=False)
    finally:
        srv.close()
    for q, r in list(zip(reqs, res))[:2]:
        s = q.shot
        _, _, ref = oracle.run(3, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width, src=s.src,
                               wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt)
        assert pl.rel_l2(r.traces, ref) <= 1e-4


def test_moving_a_model_between_streams_keeps_its_work_in_order(fdlib):
    """fd_set_stream between chunks (to streams of other priorities) gives the same
    traces and wavefield, bitwise, as one uninterrupted run."""
    shot = wl.serving_3d_shot(0, 64, 90, seed=93, sponge_width=8)
    ref = alone(fdlib, shot)
    handles = [fdlib.fd_stream_create(p)[0] for p in (0, -1, -5)]
    try:
        with fdlib.Model.from_shot(shot, stream=handles[0]) as m:
            fdlib.fd_reset(m.handle)
            fdlib.fd_set_trace_buffer(m.handle, None, shot.nt)
            for k in range(9):
                fdlib.fd_set_stream(m.handle, handles[k % 3])
                m.step(10)
            np.testing.assert_array_equal(m.traces(shot.nt), ref)
    finally:
        for h in handles:
            fdlib.fd_stream_destroy(h)


def test_one_at_a_time_and_budget(fdlib):
    from paper_2311_05038_b300 import serving
    reqs = [serving.Request(i, 0.0, s) for i, _, s in stream(n=6, seed=91)]
    fps = sorted(serving.footprint_bytes(q.shot, 200) for q in reqs)
    budget = fps[-1] + fps[-2]                     # at most two of the largest models
    srv = serving.Server(max_active=3, budget_bytes=budget, chunk=50, max_nt=200)
    try:
        res = srv.serve(reqs, realtime=False)
        assert srv.pool.peak <= budget
    finally:
        srv.close()
    one = serving.Server(max_active=1, chunk=50, max_nt=200)
    try:
        res1 = one.serve(reqs, realtime=False)
    finally:
        one.close()
    for a, b in zip(res, res1):
        np.testing.assert_array_equal(a.traces, b.traces)
    s = serving.summarize(res)
    assert s["shots"] == 6 and s["p99_s"] >= s["p50_s"] > 0
