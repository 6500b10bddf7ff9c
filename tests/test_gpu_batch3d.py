"""Batched 3D shots: one launch per time step over many models, each CTA stepping
its own model with the single-shot 3D kernel (needs a CUDA device).

The arithmetic is the single-shot step's, so every model's wavefield and traces
must equal its solo fd_run_shot bitwise, for uneven grids (tails in x, y and z,
several z chunks), sponges on and off, uneven step counts and split calls."""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def shots3d(nt=40):
    spec = [((45, 38, 70), 8), ((40, 36, 50), 0), ((33, 65, 31), 5), ((130, 70, 97), 12), ((20, 24, 28), 0),
            ((64, 64, 64), 20)]
    return [wl.roofline_3d(shape=shape, nt=nt, sponge_width=W, seed=3 + i) for i, (shape, W) in enumerate(spec)]


def solo(fd, shots, nts):
    out = []
    for s, nt in zip(shots, nts):
        with fd.Model.from_shot(s) as m:
            m.run_shot(nt)
            out.append((m.wavefield(with_old=True), m.traces(nt)))
    return out


def batched(fd, shots, nts, chunks=None):
    models = [fd.Model.from_shot(s) for s in shots]
    try:
        with fd.Batch(models) as b:
            if chunks is None:
                b.run_shots(nts)
            else:
                for m, nt in zip(models, nts):
                    fd.fd_reset(m.handle)
                    fd.fd_set_trace_buffer(m.handle, None, nt)
                for c in chunks:
                    b.step(c)
            for m, nt in zip(models, nts):
                assert fd.fd_get_step(m.handle) == nt
            return [(m.wavefield(with_old=True), m.traces(nt)) for m, nt in zip(models, nts)]
    finally:
        for m in models:
            m.close()


def assert_same(a, b):
    for (wa, ta), (wb, tb) in zip(a, b):
        np.testing.assert_array_equal(wa[0], wb[0])
        np.testing.assert_array_equal(wa[1], wb[1])
        np.testing.assert_array_equal(ta, tb)


def test_batch3d_equals_solo_bitwise_with_uneven_step_counts(fdlib):
    shots = shots3d()
    nts = [40, 17, 0, 33, 40, 25]
    assert_same(batched(fdlib, shots, nts), solo(fdlib, shots, nts))


def test_batch3d_split_calls_continue_the_run(fdlib):
    shots = shots3d(nt=30)[:4]
    nts = [30] * 4
    assert_same(batched(fdlib, shots, nts, chunks=[7, 1, 22]), solo(fdlib, shots, nts))


def test_batch3d_more_models_than_one_launch_carries(fdlib):
    """52 small models (one launch carries 48): all bitwise equal to their solo runs."""
    shots = [wl.roofline_3d(shape=(12 + i % 5, 14 + i % 3, 18 + i % 7), nt=9, sponge_width=i % 3, seed=40 + i)
             for i in range(52)]
    nts = [9 - (i % 2) for i in range(52)]
    assert_same(batched(fdlib, shots, nts), solo(fdlib, shots, nts))


def test_batch3d_matches_the_oracle(fdlib, oracle):
    shots = shots3d(nt=60)[:2]
    got = batched(fdlib, shots, [60, 60])
    for s, ((P, Pold), tr) in zip(shots, got):
        Pr, Por, trr = oracle.run(3, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width, src=s.src,
                                  wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt)
        assert max(pl.rel_l2(P, Pr), pl.rel_l2(Pold, Por), pl.rel_l2(tr, trr)) <= 1e-4


def test_batched_3d_workload_full_size(fdlib, oracle):
    """The batched 3D workload as the bench runs it (24 models, cubes 128-256, 300
    steps, one batch, z chunks chosen for the whole launch): every model equals
    its solo run bitwise, and the three 128^3 shots and one 160^3 shot match the
    FP64 oracle over the whole run (final P, Pold and traces, rel L2 <= 1e-4)."""
    shots = wl.batched_3d_shots()
    nts = [s.nt for s in shots]
    got = batched(fdlib, shots, nts)
    assert_same(got, solo(fdlib, shots, nts))
    picked = [i for i, s in enumerate(shots) if s.shape[0] == 128]
    picked.append(next(i for i, s in enumerate(shots) if s.shape[0] == 160))
    assert len(picked) == 4
    for i in picked:
        s = shots[i]
        (P, Pold), tr = got[i]
        Pr, Por, trr = oracle.run(3, s.shape, s.h, s.dt, s.vel, sponge_width=s.sponge_width, src=s.src,
                                  wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt)
        errs = (pl.rel_l2(P, Pr), pl.rel_l2(Pold, Por), pl.rel_l2(tr, trr))
        assert np.all(np.isfinite(P)) and max(errs) <= 1e-4, (s.name, errs)
