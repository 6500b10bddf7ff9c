"""Batched multi-shot launches: every shot is bitwise the same alone and in a batch.

The batch advances uneven 2D shots in one persistent launch (a table of
(shot, tile) items gated by per-tile step counters).  Its arithmetic is the
single-shot step's, so wavefields and traces must match fd_run_shot exactly
under every tile shape, group budget and steps-per-launch setting, and for
shots that stop at different steps.
"""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def small_shots(n=5, nt=120, seed=50):
    rng = np.random.default_rng(seed)
    shots = []
    for i in range(n):
        nz = int(rng.integers(40, 140))
        nx = int(rng.integers(50, 220))
        vel = wl.grf_velocity((nz, nx), corr_cells=5.0, vmin=1500.0, vmax=4000.0, seed=60 + i)
        dt = wl.courant_dt(10.0, float(vel.max()))
        rec = np.array([(ix, 0, min(12, nz - 1)) for ix in range(0, nx, 3)], np.int32)
        shots.append(wl.Shot(2, (nz, nx), 10.0, dt, nt, vel, (nx // 2, 0, nz // 2), wl.ricker(nt, dt, 25.0),
                             rec, sponge_width=8 if i % 2 == 0 else 0, name=f"batch-small-{i}"))
    return shots


def solo(fd, shots, nts):
    out = []
    for s, nt in zip(shots, nts):
        with fd.Model.from_shot(s) as m:
            m.run_shot(nt)
            out.append((m.wavefield(with_old=True), m.traces(nt)))
    return out


def batched(fd, shots, nts, tuning):
    models = [fd.Model.from_shot(s) for s in shots]
    with fd.Batch(models) as b:
        if tuning is not None:
            b.set_tuning(**tuning)
        b.run_shots(nts)
        out = [(m.wavefield(with_old=True), m.traces(nt)) for m, nt in zip(models, nts)]
    for m in models:
        m.close()
    return out


def assert_same(a, b):
    for (wa, ta), (wb, tb) in zip(a, b):
        np.testing.assert_array_equal(wa[0], wb[0])
        np.testing.assert_array_equal(wa[1], wb[1])
        np.testing.assert_array_equal(ta, tb)


@pytest.mark.parametrize("tuning", [
    dict(tile=0, steps_per_launch=2000, ctas_per_sm=0, group_mb=0),
    dict(tile=1, steps_per_launch=37, ctas_per_sm=0, group_mb=0),
    dict(tile=2, steps_per_launch=50, ctas_per_sm=1, group_mb=1),
    dict(tile=0, steps_per_launch=7, ctas_per_sm=2, group_mb=1),
    dict(tile=3, steps_per_launch=2000, ctas_per_sm=0, group_mb=0),
    dict(tile=4, steps_per_launch=2000, ctas_per_sm=0, group_mb=1),
    dict(tile=5, steps_per_launch=2000, ctas_per_sm=0, group_mb=0),
    dict(tile=6, steps_per_launch=2000, ctas_per_sm=0, group_mb=1),
    dict(tile=7, steps_per_launch=2000, ctas_per_sm=0, group_mb=0),
])
def test_batch_equals_solo_bitwise(fdlib, tuning):
    shots = small_shots()
    nts = [s.nt for s in shots]
    assert_same(batched(fdlib, shots, nts, tuning), solo(fdlib, shots, nts))


@pytest.mark.parametrize("tile", [0, 3, 6])
def test_batch_uneven_step_counts(fdlib, tile):
    shots = small_shots(n=4, nt=90, seed=51)
    nts = [90, 17, 0, 64]
    ref = solo(fdlib, shots, nts)
    got = batched(fdlib, shots, nts, dict(tile=tile, steps_per_launch=25, ctas_per_sm=0, group_mb=0))
    assert_same(got, ref)


def test_wide_schedule_splits_many_shots_over_launches(fdlib):
    """More shots than one wide launch carries (64): every shot still bitwise equal to its solo run."""
    shots = small_shots(n=70, nt=12, seed=55)
    nts = [12 - (i % 3) for i in range(70)]
    assert_same(batched(fdlib, shots, nts, dict(tile=3, steps_per_launch=1, ctas_per_sm=0, group_mb=0)),
                solo(fdlib, shots, nts))


def test_batch_matches_oracle(fdlib, oracle):
    shots = small_shots(n=3, nt=150, seed=52)
    got = batched(fdlib, shots, [s.nt for s in shots], None)
    for s, ((P, Pold), tr) in zip(shots, got):
        Pr, Poldr, trr = oracle.run(2, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width, src=s.src,
                                    wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt)
        assert pl.rel_l2(P, Pr) <= 1e-4 and pl.rel_l2(Pold, Poldr) <= 1e-4 and pl.rel_l2(tr, trr) <= 1e-4


@pytest.mark.parametrize("tile", [1, 3])
def test_batch_step_continues_a_run(fdlib, tile):
    """Two batch calls of 30 + 45 steps equal one solo run of 75."""
    shots = small_shots(n=3, nt=75, seed=53)
    ref = solo(fdlib, shots, [75, 75, 75])
    models = [fdlib.Model.from_shot(s) for s in shots]
    with fdlib.Batch(models) as b:
        b.set_tuning(tile=tile, steps_per_launch=16, ctas_per_sm=0, group_mb=0)
        for m in models:
            fdlib.fd_reset(m.handle)
            fdlib.fd_set_trace_buffer(m.handle, None, 75)
        b.step(30)
        b.step(45)
        got = [(m.wavefield(with_old=True), m.traces(75)) for m in models]
        assert all(fdlib.fd_get_step(m.handle) == 75 for m in models)
    assert_same(got, ref)


def test_autotune_picks_a_valid_tuning(fdlib):
    """The tuner's choice is one of its candidates: a persistent schedule keeps the
    caller's 2000 steps per launch unless a launch of 5 or 2 of the 10 trial
    steps was faster; the wide schedules keep it unused.  Results stay those of
    the solo runs."""
    shots = small_shots(n=4, nt=60, seed=54)
    models = [fdlib.Model.from_shot(s) for s in shots]
    with fdlib.Batch(models) as b:
        best = b.autotune(trial_steps=10)
        assert best["tile"] in range(8)
        assert best["steps_per_launch"] in ((2000, 5, 2) if best["tile"] < 3 else (2000,))
        assert b.tuning() == best
        b.run_shots([60] * 4)
        got = [(m.wavefield(with_old=True), m.traces(60)) for m in models]
    assert_same(got, solo(fdlib, shots, [60] * 4))


def test_autotune_steps_per_launch_candidates(fdlib):
    """With the caller's steps per launch (3) shorter than the trial (12), the
    persistent candidates are 12, 6 and 3 steps per launch; whichever wins, a
    run in launches of that length equals the solo runs bitwise."""
    shots = small_shots(n=3, nt=50, seed=57)
    models = [fdlib.Model.from_shot(s) for s in shots]
    with fdlib.Batch(models) as b:
        b.set_tuning(tile=0, steps_per_launch=3, ctas_per_sm=0, group_mb=0)
        best = b.autotune(trial_steps=12)
        assert best["steps_per_launch"] in ((12, 6, 3) if best["tile"] < 3 else (3,))
        b.run_shots([50] * 3)
        got = [(m.wavefield(with_old=True), m.traces(50)) for m in models]
    assert_same(got, solo(fdlib, shots, [50] * 3))
    # the same shapes from a longer starting launch are tuned afresh, not served
    # from the cache entry above: a 12-step winner now keeps 2000
    with fdlib.Batch(models) as b:
        b.set_tuning(tile=0, steps_per_launch=2000, ctas_per_sm=0, group_mb=0)
        best2 = b.autotune(trial_steps=12)
        assert best2["steps_per_launch"] in ((2000, 6, 3) if best2["tile"] < 3 else (2000,))
    for m in models:
        m.close()


def test_batch_rejects_a_mix_of_2d_and_3d_models(fdlib):
    shot = wl.roofline_3d(shape=(16, 16, 16), nt=4, sponge_width=0)
    with fdlib.Model.from_shot(shot) as m, fdlib.Model.from_shot(small_shots(n=1)[0]) as m2:
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_batch_create([m.handle, m2.handle])
        assert e.value.status == fdlib.FD_EINVAL


def test_stalled_item_times_out_and_context_survives(fdlib):
    """A tile whose completion is withheld makes its neighbours' bounded waits run
    out: fd_batch_step returns FD_ETIMEOUT (no fault, no hang), and the same
    context then runs a clean batch whose results equal the solo runs."""
    import time
    shots = small_shots(n=3, nt=40, seed=55)
    models = [fdlib.Model.from_shot(s) for s in shots]
    with fdlib.Batch(models) as b:
        b.set_tuning(tile=0, steps_per_launch=40, ctas_per_sm=0, group_mb=0)
        fdlib.fd_batch_set_fault(b.handle, 1)
        t0 = time.perf_counter()
        with pytest.raises(fdlib.FDError) as e:
            b.run_shots([40, 40, 40])
        assert e.value.status == fdlib.FD_ETIMEOUT
        assert time.perf_counter() - t0 < 30
        fdlib.fd_batch_set_fault(b.handle, -1)
        b.run_shots([40, 40, 40])
        got = [(m.wavefield(with_old=True), m.traces(40)) for m in models]
    for m in models:
        m.close()
    assert_same(got, solo(fdlib, shots, [40, 40, 40]))


@pytest.mark.parametrize("tile", [0, 6])
def test_batched_workload_full_size_vs_oracle(fdlib, oracle, tile):
    """The 64-shot batched workload at its full grid sizes, every shot started from a
    random state so that every tile is active, 10 steps in one batch (the persistent
    schedule, and the wide one with columns of 8 tiles); six shots (the
    smallest, the largest and four seeded others) against the oracle, rel L2 <= 1e-4
    for both levels and the traces."""
    nt = 10
    shots = [wl.batched_2d_shot(i, s, nt) for i, s in enumerate(wl.batched_2d_shapes(64))]
    states = [wl.random_state(s.shape, seed=900 + i) for i, s in enumerate(shots)]
    models = [fdlib.Model.from_shot(s) for s in shots]
    try:
        for m, (P0, Pm1) in zip(models, states):
            fdlib.fd_set_wavefield(m.handle, P0, Pm1, 0)
            fdlib.fd_set_trace_buffer(m.handle, None, nt)
        with fdlib.Batch(models) as b:
            b.set_tuning(tile=tile, steps_per_launch=2000, ctas_per_sm=0, group_mb=96 if tile < 3 else 0)
            b.step(nt)
        sizes = [s.npoints for s in shots]
        pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
        pick |= set(np.random.default_rng(3).choice(64, 4, replace=False).tolist())
        for i in sorted(pick):
            s = shots[i]
            (P, Pold), tr = models[i].wavefield(with_old=True), models[i].traces(nt)
            rP, rPold, rtr = oracle.run(2, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width,
                                        sponge_R=s.sponge_R, src=s.src, wavelet=s.wavelet, receivers=s.receivers,
                                        P=states[i][0], Pold=states[i][1], nsteps=nt)
            errs = (pl.rel_l2(P, rP), pl.rel_l2(Pold, rPold), pl.rel_l2(tr, rtr))
            assert max(errs) <= 1e-4, (i, s.shape, errs)
    finally:
        for m in models:
            m.close()
