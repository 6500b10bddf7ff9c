"""The C example (a 3D shot through include/fd.h alone) on the GPU: its traces
match the FP64 oracle and the Python binding's run of the same shot."""
import subprocess

import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available
from test_abi_cpu import _build_c_example

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def _same_shot():
    """The shot example_shot.c builds, restated here."""
    nx, ny, nz, nt, W, stride = 96, 80, 64, 300, 10, 4
    h = 10.0
    dt = 0.4 * h / 3000.0
    vel = np.empty((nz, ny, nx), np.float32)
    for z in range(nz):
        vel[z] = 1800.0 if z < nz // 3 else 2400.0 if z < 2 * nz // 3 else 3000.0
    rec = np.array([(ix, iy, W + 3) for iy in range(0, ny, stride) for ix in range(0, nx, stride)], np.int32)
    return wl.Shot(3, (nz, ny, nx), h, dt, nt, vel, (nx // 2, ny // 2, W + 6), wl.ricker(nt, dt, 15.0), rec,
                   sponge_width=W)


def test_c_example_runs_and_matches(fdlib, oracle, tmp_path):
    exe = _build_c_example(tmp_path)
    out = tmp_path / "traces.bin"
    r = subprocess.run([exe, str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    shot = _same_shot()
    got = np.fromfile(out, dtype=np.float32).reshape(shot.nt, len(shot.receivers))
    with fdlib.Model.from_shot(shot) as m:
        m.run_shot(shot.nt)
        py = m.traces(shot.nt)
    _, _, ref = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                           src=shot.src, wavelet=shot.wavelet, receivers=shot.receivers, nsteps=shot.nt)
    assert pl.rel_l2(got, ref) <= 1e-4
    assert pl.rel_l2(got, py) <= 1e-6       # the same library; the wavelets may differ in the last ulp
