"""The allocation-free batch entry point gives the same results as fd_batch_step.

fd_batch_step_noalloc is meant for callers that cannot allocate device memory
once they are running (a serving process whose pool already holds the device
memory, or a loop that must avoid cudaMalloc's device-wide synchronisation).
It runs the persistent batch kernel with its scratch in a static device array.
This file is collected last on purpose.  It checks two consecutive calls against
the allocating entry point, within the tolerance of the parity tests (relative
L2 1e-4); the results are in fact bitwise identical.  Each call clears the shared
array's counters, so a second call must not see the first one's leftovers.
"""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

TOL = 1e-4


def shots(n=3, nt=100, seed=70):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nz = int(rng.integers(40, 130))
        nx = int(rng.integers(60, 200))
        vel = wl.grf_velocity((nz, nx), corr_cells=5.0, vmin=1500.0, vmax=4000.0, seed=80 + i)
        dt = wl.courant_dt(10.0, float(vel.max()))
        rec = np.array([(ix, 0, min(10, nz - 1)) for ix in range(0, nx, 5)], np.int32)
        out.append(wl.Shot(2, (nz, nx), 10.0, dt, nt, vel, (nx // 2, 0, nz // 2), wl.ricker(nt, dt, 25.0), rec,
                           sponge_width=6 if i != 1 else 0))
    return out


def fresh_models(fd, ss, nt):
    models = [fd.Model.from_shot(s) for s in ss]
    for m in models:
        fd.fd_reset(m.handle)
        fd.fd_set_trace_buffer(m.handle, None, nt)
    return models


def state(models, nt):
    return [(m.wavefield(with_old=True), m.traces(nt)) for m in models]


def assert_close(got, ref):
    for ((P, Po), tr), ((Pr, Por), trr) in zip(got, ref):
        assert pl.rel_l2(P, Pr) <= TOL and pl.rel_l2(Po, Por) <= TOL and pl.rel_l2(tr, trr) <= TOL


def test_no_alloc_matches_batch_step_on_two_calls(fdlib):
    nt = 100
    ss = shots(nt=nt)
    # reference: the allocating batch entry point, same two calls
    ref_models = fresh_models(fdlib, ss, nt)
    with fdlib.Batch(ref_models) as b:
        b.step(40)
        ref_first = state(ref_models, nt)
        b.step(35)
        ref_second = state(ref_models, nt)
    models = fresh_models(fdlib, ss, nt)
    handles = [m.handle for m in models]
    fdlib.fd_batch_step_noalloc(handles, 40)
    assert_close(state(models, nt), ref_first)
    fdlib.fd_batch_step_noalloc(handles, 35)
    assert_close(state(models, nt), ref_second)
    assert all(fdlib.fd_get_step(h) == 75 for h in handles)
    for m in models + ref_models:
        m.close()


def test_no_alloc_second_call_on_other_models_ignores_leftovers(fdlib, oracle):
    """One call on three models leaves its descriptors, tile table and receiver
    lists in the shared array; a following call on two other models, with other
    grids, receiver counts and sponge settings, must match both the allocating
    batch entry point and the oracle."""
    nt = 60
    first = shots(n=3, nt=nt, seed=71)
    models = fresh_models(fdlib, first, nt)
    fdlib.fd_batch_step_noalloc([m.handle for m in models], nt)
    for m in models:
        m.close()
    second = []
    for i, (nz, nx, W) in enumerate(((37, 91, 0), (70, 45, 5))):
        vel = wl.grf_velocity((nz, nx), corr_cells=4.0, vmin=1500.0, vmax=3500.0, seed=90 + i)
        dt = wl.courant_dt(10.0, float(vel.max()))
        rec = np.array([(ix, 0, iz) for iz in (3, nz - 4) for ix in range(1, nx, 7 + i)], np.int32)
        second.append(wl.Shot(2, (nz, nx), 10.0, dt, nt, vel, (nx // 3, 0, nz // 2), wl.ricker(nt, dt, 30.0), rec,
                              sponge_width=W))
    ref_models = fresh_models(fdlib, second, nt)
    with fdlib.Batch(ref_models) as b:
        b.step(nt)
        ref = state(ref_models, nt)
    models = fresh_models(fdlib, second, nt)
    fdlib.fd_batch_step_noalloc([m.handle for m in models], nt)
    got = state(models, nt)
    assert_close(got, ref)
    for s, ((P, Po), tr) in zip(second, got):
        Pr, Por, trr = oracle.run(2, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width, src=s.src,
                                  wavelet=s.wavelet, receivers=s.receivers, nsteps=nt)
        assert pl.rel_l2(P, Pr) <= TOL and pl.rel_l2(Po, Por) <= TOL and pl.rel_l2(tr, trr) <= TOL
    for m in models + ref_models:
        m.close()


def test_no_alloc_rejects_requests_beyond_its_limits(fdlib):
    ss = shots(n=1, nt=4)
    with fdlib.Model.from_shot(ss[0]) as m:
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_batch_step_noalloc([m.handle] * 65, 1)
        assert e.value.status == fdlib.FD_EBUDGET
        big = wl.Shot(2, (4112, 8192), 10.0, 0.001, 4, np.full((4112, 8192), 2000.0, np.float32), (5, 0, 5),
                      wl.ricker(4, 0.001, 20.0), np.zeros((0, 3), np.int32))
        with fdlib.Model.from_shot(big) as mb:
            with pytest.raises(fdlib.FDError) as e:
                fdlib.fd_batch_step_noalloc([mb.handle], 1)
            assert e.value.status == fdlib.FD_EBUDGET
            assert "static limit" in fdlib.fd_last_error()
