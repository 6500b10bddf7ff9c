"""Two time steps per launch (fd_set_time_fusion) against single steps and the
oracle (needs a CUDA device).

The fused launch evaluates the paper's damped leapfrog (section 7, Eq. 1) twice
per point with the single-step kernel's arithmetic, so its levels and traces
must equal those of single steps bitwise, for any grid shape, sponge, source
position and step count (an odd count ends with one single step)."""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def run(fd, shot, nt, fuse, chunks=None, P0=None, Pm1=None):
    with fd.Model.from_shot(shot) as m:
        if fuse:
            m.set_time_fusion(2)
        if P0 is None:
            if chunks is None:
                m.run_shot(nt)
            else:
                fd.fd_reset(m.handle)
                fd.fd_set_trace_buffer(m.handle, None, nt)
                for c in chunks:
                    m.step(c)
        else:
            fd.fd_set_trace_buffer(m.handle, None, nt)
            fd.fd_set_wavefield(m.handle, P0, Pm1, 0)
            m.step(nt)
        assert fd.fd_get_step(m.handle) == nt
        P, Po = m.wavefield(with_old=True)
        return P, Po, m.traces(nt)


def assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("shape,W,nt", [((45, 38, 70), 8, 61), ((40, 36, 50), 7, 40), ((9, 11, 13), 0, 17),
                                        ((33, 65, 31), 5, 30), ((130, 70, 97), 12, 25)])
def test_fused_pairs_equal_single_steps_bitwise(fdlib, shape, W, nt):
    """Ragged grids (tails in x, y and z; several z chunks at 130 planes), sponge
    on and off, odd and even step counts."""
    shot = wl.roofline_3d(shape=shape, nt=nt, sponge_width=W)
    assert_same(run(fdlib, shot, nt, True), run(fdlib, shot, nt, False))


def test_fused_pairs_from_a_random_state_full_size(fdlib):
    """512^3 (the benchmark grid and launch geometry), every point active from a
    random state, 4 steps with the source on."""
    shot = wl.roofline_3d(n=512, nt=4)
    P0, Pm1 = wl.random_state(shot.shape, seed=51)
    assert_same(run(fdlib, shot, 4, True, P0=P0, Pm1=Pm1), run(fdlib, shot, 4, False, P0=P0, Pm1=Pm1))


def test_fused_pairs_in_split_calls(fdlib):
    """Calls of odd and even lengths interleave fused pairs and single steps; every
    receiver row is still recorded exactly once."""
    shot = wl.roofline_3d(shape=(40, 36, 50), nt=30, sponge_width=7)
    assert_same(run(fdlib, shot, 30, True, chunks=[3, 4, 1, 2, 7, 13]), run(fdlib, shot, 30, False))


def test_fused_pairs_match_the_oracle(fdlib, oracle):
    """The layered workload at 96^3 with a 20-point sponge, 400 steps in fused pairs,
    against the FP64 oracle (rel L2 <= 1e-4)."""
    shot = wl.roofline_3d(n=96, nt=400, sponge_width=20)
    P, Po, tr = run(fdlib, shot, shot.nt, True)
    Pr, Por, trr = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                              src=shot.src, wavelet=shot.wavelet, receivers=shot.receivers, nsteps=shot.nt)
    assert max(pl.rel_l2(P, Pr), pl.rel_l2(Po, Por), pl.rel_l2(tr, trr)) <= 1e-4


def test_time_fusion_arguments(fdlib):
    shot2 = wl.parity_2d(nt=2)
    with fdlib.Model.from_shot(shot2) as m:
        with pytest.raises(fdlib.FDError) as e:
            m.set_time_fusion(2)
        assert e.value.status == fdlib.FD_EINVAL
        m.set_time_fusion(1)
    shot = wl.roofline_3d(shape=(12, 12, 12), nt=2, sponge_width=0)
    with fdlib.Model.from_shot(shot) as m:
        for bad in (0, 3, -1):
            with pytest.raises(fdlib.FDError):
                m.set_time_fusion(bad)
