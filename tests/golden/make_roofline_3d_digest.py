"""Write the FP64 oracle's digest of the full 3D roofline shot.

The shot is the layered 512^3 workload with a 20-point sponge, a 10 Hz Ricker
source near the top and 256 x 256 receivers, run for all 1000 steps (the paper's
Eq. 1 advanced by the scheme of section 7).  Its outputs (two 1 GB FP64
wavefield levels and 65 536 x 1000 traces) are too large to store, so this
script keeps what a GPU test needs to compare a full run with it:

* the FP64 L2 norms and CountSketches (``tests/digest.py``) of the final P, the
  final Pold and the whole trace array;
* exact values, rounded to FP32 (relative rounding <= 6e-8 per element), of the
  final P on the vertical plane through the source (iy = 256, all 512 x 512
  points) and of the 1000-sample traces of the 256 receivers on the row
  through the source.

It calls only the oracle and the seeded input generators.  The oracle runs in
chunks of 50 steps (its n0 argument keeps the source's time index), which is
the same recurrence as one call.  On 8 host cores it takes about half an hour.

Usage: ``python tests/golden/make_roofline_3d_digest.py [--threads N]``.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import digest  # noqa: E402  (tests/digest.py)
import workloads as wl  # noqa: E402
from oracle import oracle  # noqa: E402

OUT = os.path.join(HERE, "roofline_3d_512_1000steps_oracle.npz")
CHUNK_STEPS = 50


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    shot = wl.roofline_3d(n=a.n, nt=a.nt)
    nz, ny, nx = shot.shape
    P = np.zeros(shot.shape)
    Pold = np.zeros(shot.shape)
    traces = np.zeros((shot.nt, len(shot.receivers)))
    t0 = time.time()
    for n0 in range(0, shot.nt, CHUNK_STEPS):
        k = min(CHUNK_STEPS, shot.nt - n0)
        P, Pold, tr = oracle.run(3, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                                 sponge_R=shot.sponge_R, src=shot.src, wavelet=shot.wavelet,
                                 receivers=shot.receivers, P=P, Pold=Pold, n0=n0, nsteps=k,
                                 nthreads=a.threads)
        traces[n0:n0 + k] = tr
        el = time.time() - t0
        print(f"steps {n0 + k}/{shot.nt}  {el:.0f} s  "
              f"{(n0 + k) * shot.npoints / el / 1e9:.3f} Gupd/s", flush=True)
    (nP, nPold), (yP, yPold) = digest.sketch([P, Pold])
    (ntr,), (ytr,) = digest.sketch([traces])
    sy = shot.src[1]
    row = np.nonzero(shot.receivers[:, 1] == sy)[0]
    np.savez_compressed(
        a.out, name=shot.name, shape=np.array(shot.shape), nt=shot.nt, src=np.array(shot.src),
        sketch_k=16384, sketch_seed=0x5EED,
        norm_P=nP, norm_Pold=nPold, norm_traces=ntr,
        sketch_P=yP, sketch_Pold=yPold, sketch_traces=ytr,
        plane_iy=sy, plane_P=P[:, sy, :].astype(np.float32),
        row_receivers=row.astype(np.int32), row_traces=traces[:, row].astype(np.float32),
        oracle_seconds=time.time() - t0, oracle_threads=oracle.max_threads() if a.threads == 0 else a.threads)
    print("wrote", a.out, f"norms P {nP:.6e} Pold {nPold:.6e} traces {ntr:.6e}")


if __name__ == "__main__":
    main()
