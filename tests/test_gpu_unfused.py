"""The paper's unfused routine sequence (add_source, fd_pzz, fd_pxx, fd_time, swap)
against the oracle and against the fused step (needs a CUDA device)."""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

TOL = 1e-4


def run(fd, shot, nt, unfused):
    with fd.Model.from_shot(shot) as m:
        fd.fd_reset(m.handle)
        fd.fd_set_trace_buffer(m.handle, None, nt)
        (fd.fd_step_unfused if unfused else fd.fd_step)(m.handle, nt)
        return m.wavefield(with_old=True), m.traces(nt)


@pytest.mark.parametrize("shot", [wl.parity_2d(nt=300), wl.roofline_3d(shape=(40, 36, 70), nt=200, sponge_width=8),
                                  wl.roofline_3d(shape=(150, 70, 45), nt=40, sponge_width=6)],
                         ids=["2d", "3d", "3d-long-axes"])
def test_unfused_matches_oracle_and_fused(fdlib, oracle, shot):
    (P, Pold), tr = run(fdlib, shot, shot.nt, unfused=True)
    Pr, Poldr, trr = oracle.run(shot.ndim, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                                src=shot.src, wavelet=shot.wavelet, receivers=shot.receivers, nsteps=shot.nt)
    assert pl.rel_l2(P, Pr) <= TOL and pl.rel_l2(Pold, Poldr) <= TOL and pl.rel_l2(tr, trr) <= TOL
    (Pf, _), trf = run(fdlib, shot, shot.nt, unfused=False)
    assert pl.rel_l2(P, Pf) <= 1e-5 and pl.rel_l2(tr, trf) <= 1e-5


def test_routine_sequence_by_hand_equals_step_unfused(fdlib):
    shot = wl.roofline_3d(shape=(24, 20, 36), nt=6, sponge_width=4)
    a = run(fdlib, shot, 6, unfused=True)
    with fdlib.Model.from_shot(shot) as m:
        fdlib.fd_reset(m.handle)
        fdlib.fd_set_trace_buffer(m.handle, None, 6)
        for _ in range(6):
            for r in (fdlib.FD_ROUTINE_PXX, fdlib.FD_ROUTINE_PYY, fdlib.FD_ROUTINE_PZZ, fdlib.FD_ROUTINE_TIME,
                      fdlib.FD_ROUTINE_ADD_SOURCE, fdlib.FD_ROUTINE_SWAP):
                fdlib.fd_routine(m.handle, r)
        b = (m.wavefield(with_old=True), m.traces(6))
    np.testing.assert_array_equal(a[0][0], b[0][0])
    np.testing.assert_array_equal(a[1], b[1])


def test_pyy_on_2d_is_einval(fdlib):
    with fdlib.Model.from_shot(wl.parity_2d(nt=2)) as m:
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_routine(m.handle, fdlib.FD_ROUTINE_PYY)
        assert e.value.status == fdlib.FD_EINVAL
