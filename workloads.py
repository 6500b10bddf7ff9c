"""Seeded synthetic inputs for the acoustic FD propagator.

This module holds no arithmetic of the propagation method.  It only draws the
inputs that both the CUDA library and the FP64 oracle consume, so that both see
the same bytes: velocity models (FP32, m/s), the Ricker source signature S(t)
(FP32), the time step chosen at a Courant number, and source / receiver grid
points.  Arrays are x-fastest: 2D ``[nz][nx]``, 3D ``[nz][ny][nx]``.  Points are
``(ix, iy, iz)`` triples; iy is 0 in 2D.

Workload recipes (the paper prints no problem sizes; these follow the stated
benchmark configurations, every random draw seeded):

* ``parity_2d``: 256 x 256, h = 10 m, v = 2000 m/s, dt at Courant 0.4 (2 ms),
  500 steps, 15 Hz Ricker at the centre, 64 receivers every 4th point of row
  iz = 64, zero-halo boundaries, no sponge.
* ``roofline_3d``: n^3 (n = 512), h = 10 m, 10 flat layers with boundaries at
  ``floor(k n / 10)`` and velocities i.i.d. U(1500, 4500) (seed 1, unsorted),
  dt at Courant 0.4 of the drawn maximum, 20-point sponge on all faces, 1000
  steps, 10 Hz Ricker at (n/2, n/2, W + 10), receivers on plane iz = W + 5 over
  ix, iy in [n/4, 3n/4) (256 x 256 at n = 512).
* ``batched_2d``: 64 shots; seed 2 draws nx from {512, 576, ..., 2048} and nz from
  {512, ..., 1024}; velocity = white noise (seed 3 + shot) smoothed by a
  Gaussian of 20 cells (200 m) and mapped affinely onto [1500, 4000]; 2000 steps.
* ``serving_3d``: a Poisson stream of shots (seed 4) with cubes n in
  {128, 160, ..., 384} and nt in [200, 2000]; velocity = the layered model plus
  500 m/s times a product of three 1D Gaussian random fields (200 m), clipped
  to [1500, 4500]; dt at Courant 0.4 of 4500 m/s.
* ``adjoint_3d``: 256^3 smoothed random velocity in [1500, 4000] (seed 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

COURANT = 0.4


@dataclass
class Shot:
    """One propagation problem: grid, model, source and receivers."""
    ndim: int
    shape: tuple            # (nz, nx) or (nz, ny, nx)
    h: float
    dt: float
    nt: int
    vel: np.ndarray         # FP32, shape
    src: tuple              # (ix, iy, iz)
    wavelet: np.ndarray     # FP32 [nt], S(t_n) at t_n = n dt
    receivers: np.ndarray   # int32 [nrec, 3] of (ix, iy, iz)
    sponge_width: int = 0
    sponge_R: float = 1e-3
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nx(self):
        return self.shape[-1]

    @property
    def ny(self):
        return self.shape[1] if self.ndim == 3 else 1

    @property
    def nz(self):
        return self.shape[0]

    @property
    def npoints(self):
        return int(np.prod(self.shape))


def ricker(nt: int, dt: float, f: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of unit peak, delayed by t0 = 1.5 / f, sampled at n dt (FP32)."""
    if t0 is None:
        t0 = 1.5 / f
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f * (t - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def courant_dt(h: float, v_max: float, courant: float = COURANT) -> float:
    """Time step giving Courant number v_max dt / h = courant."""
    return courant * h / v_max


def layered_velocity(shape, nlayers: int = 10, vmin: float = 1500.0, vmax: float = 4500.0,
                     seed: int = 1) -> np.ndarray:
    """Flat layers along z, boundaries at floor(k nz / nlayers), v ~ U(vmin, vmax)."""
    rng = np.random.default_rng(seed)
    vl = rng.uniform(vmin, vmax, nlayers)
    nz = shape[0]
    bounds = [(k * nz) // nlayers for k in range(nlayers + 1)]
    col = np.empty(nz, dtype=np.float64)
    for k in range(nlayers):
        col[bounds[k]:bounds[k + 1]] = vl[k]
    v = np.empty(shape, dtype=np.float32)
    v[...] = col.reshape((nz,) + (1,) * (len(shape) - 1)).astype(np.float32)
    return v


def random_field(shape, corr_cells: float, seed: int) -> np.ndarray:
    """White noise N(0,1) smoothed by a Gaussian of std corr_cells (FFT, periodic), FP64."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    spec = np.fft.rfftn(noise)
    freqs = np.meshgrid(*[np.fft.fftfreq(n) for n in shape[:-1]],
                        np.fft.rfftfreq(shape[-1]), indexing="ij")
    k2 = sum(f * f for f in freqs)
    spec *= np.exp(-2.0 * (math.pi ** 2) * (corr_cells ** 2) * k2)
    return np.fft.irfftn(spec, s=shape, axes=tuple(range(len(shape))))


def grf_velocity(shape, corr_cells: float = 20.0, vmin: float = 1500.0, vmax: float = 4000.0,
                 seed: int = 3) -> np.ndarray:
    """Smoothed random field mapped affinely onto [vmin, vmax] (FP32)."""
    g = random_field(shape, corr_cells, seed)
    g = (g - g.min()) / max(g.max() - g.min(), 1e-300)
    return (vmin + (vmax - vmin) * g).astype(np.float32)


def random_state(shape, seed: int, scale: float = 1.0):
    """Two independent N(0, scale^2) FP32 fields, used as initial (P, Pold)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape).astype(np.float32) * scale,
            rng.standard_normal(shape).astype(np.float32) * scale)


def device_random_fields(shape, seed: int, vmin: float = 1500.0, vmax: float = 2500.0, device="cuda"):
    """(vel, P, Pold) as FP32 torch tensors generated on the device from one seeded
    generator: vel ~ U(vmin, vmax), P and Pold ~ N(0, 1).  For grids too large to
    generate and upload from the host in a test (billions of points)."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    vel = torch.rand(shape, device=device, generator=g).mul_(vmax - vmin).add_(vmin)
    P = torch.randn(shape, device=device, generator=g)
    Pold = torch.randn(shape, device=device, generator=g)
    return vel, P, Pold


# ------------------------------------------------------------------------ workloads

def parity_2d(nt: int = 500) -> Shot:
    """256 x 256 constant-velocity 2D shot (the FP32-vs-FP64 parity workload)."""
    n, h, v0, f = 256, 10.0, 2000.0, 15.0
    dt = courant_dt(h, v0)
    vel = np.full((n, n), v0, dtype=np.float32)
    rec = np.array([(ix, 0, 64) for ix in range(0, 256, 4)], dtype=np.int32)
    return Shot(ndim=2, shape=(n, n), h=h, dt=dt, nt=nt, vel=vel, src=(128, 0, 128),
                wavelet=ricker(nt, dt, f), receivers=rec, sponge_width=0,
                name=f"2d-256x256-const2000-r4-{nt}steps")


def roofline_3d(n: int = 512, nt: int = 1000, sponge_width: int = 20, seed: int = 1,
                shape=None) -> Shot:
    """Layered 3D shot; n = 512, nt = 1000 is the single-shot roofline workload.

    ``shape`` (nz, ny, nx) overrides the cube for ragged parity cases; positions
    scale with the grid.
    """
    if shape is None:
        shape = (n, n, n)
    nz, ny, nx = shape
    h, f = 10.0, 10.0
    vel = layered_velocity(shape, seed=seed)
    dt = courant_dt(h, float(vel.max()))
    W = sponge_width
    src = (nx // 2, ny // 2, min(W + 10, nz - 1))
    iz_r = min(W + 5, nz - 1)
    xs = range(nx // 4, nx // 4 + max(nx // 2, 1))
    ys = range(ny // 4, ny // 4 + max(ny // 2, 1))
    rec = np.array([(ix, iy, iz_r) for iy in ys for ix in xs], dtype=np.int32)
    return Shot(ndim=3, shape=tuple(shape), h=h, dt=dt, nt=nt, vel=vel, src=src,
                wavelet=ricker(nt, dt, f), receivers=rec, sponge_width=W,
                name=f"3d-{nz}x{ny}x{nx}-layered-r4-sponge{W}-{nt}steps")


def batched_2d_shapes(nshots: int = 64, seed: int = 2):
    """(nz, nx) per shot, nx in {512..2048}, nz in {512..1024}, multiples of 64."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(512 // 64, 2048 // 64 + 1, nshots) * 64
    nzs = rng.integers(512 // 64, 1024 // 64 + 1, nshots) * 64
    return [(int(z), int(x)) for z, x in zip(nzs, nxs)]


def batched_2d_shot(i: int, shape, nt: int = 2000, sponge_width: int = 20) -> Shot:
    """Shot i of the batched 2D workload (GRF velocity, seed 3 + i)."""
    nz, nx = shape
    h, f = 10.0, 15.0
    vel = grf_velocity(shape, corr_cells=20.0, vmin=1500.0, vmax=4000.0, seed=3 + i)
    dt = courant_dt(h, float(vel.max()))
    rec = np.array([(ix, 0, 32) for ix in range(0, nx, 4)], dtype=np.int32)
    return Shot(ndim=2, shape=(nz, nx), h=h, dt=dt, nt=nt, vel=vel, src=(nx // 2, 0, nz // 2),
                wavelet=ricker(nt, dt, f), receivers=rec, sponge_width=sponge_width,
                name=f"2d-{nz}x{nx}-grf-shot{i}")


def batched_2d(nshots: int = 64, nt: int = 2000, seed: int = 2):
    """The batched 2D workload: a list of uneven 2D shots."""
    return [batched_2d_shot(i, s, nt) for i, s in enumerate(batched_2d_shapes(nshots, seed))]


def serving_3d_stream(nshots: int = 500, seed: int = 4, rate: float = 1.0,
                      sizes=tuple(range(128, 385, 32)), nt_range=(200, 2000)):
    """Poisson arrival times (s) and per-shot (n, nt) for the serving workload."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, nshots)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = rng.choice(np.array(sizes), nshots)
    nts = rng.integers(nt_range[0], nt_range[1] + 1, nshots)
    return [(float(a), int(n), int(t)) for a, n, t in zip(arrivals, ns, nts)]


def smooth_profile(n: int, corr_cells: float, seed: int) -> np.ndarray:
    """1D white noise smoothed by a Gaussian of std corr_cells, scaled to max |.| = 1 (FP64)."""
    g = random_field((n,), corr_cells, seed)
    return g / max(np.abs(g).max(), 1e-300)


def serving_3d_velocity(n: int, seed: int, sponge_width: int = 20) -> np.ndarray:
    """Layered model (10 flat layers, U(1500, 4500)) plus a smooth random perturbation,
    clipped to [1500, 4500] (FP32).  The perturbation is 500 m/s times the product of
    three independent 1D Gaussian random fields of correlation length 200 m (20 cells),
    which keeps generation O(n^3) elementwise for the large stream of serving shots."""
    shape = (n, n, n)
    lay = layered_velocity(shape, seed=seed)
    gz = smooth_profile(n, 20.0, seed + 11)[:, None, None]
    gy = smooth_profile(n, 20.0, seed + 12)[None, :, None]
    gx = smooth_profile(n, 20.0, seed + 13)[None, None, :]
    v = lay.astype(np.float64) + 500.0 * gz * gy * gx
    return np.clip(v, 1500.0, 4500.0).astype(np.float32)


def serving_3d_shot(i: int, n: int, nt: int, seed: int = 4, sponge_width: int = 20, vel=None,
                    src_jitter: bool = True) -> Shot:
    """Shot i of the serving workload on an n^3 grid: 10 Hz source near the top (its
    x, y position drawn per shot), receivers every 2nd point of plane iz = W + 5 over
    the central half."""
    shape = (n, n, n)
    if vel is None:
        vel = serving_3d_velocity(n, seed * 1000 + i, sponge_width)
    h, f = 10.0, 10.0
    dt = courant_dt(h, 4500.0)      # one dt for the stream: Courant 0.4 at the clip velocity
    rng = np.random.default_rng(seed * 7919 + i)
    cx = n // 2 + (int(rng.integers(-n // 8, n // 8 + 1)) if src_jitter else 0)
    cy = n // 2 + (int(rng.integers(-n // 8, n // 8 + 1)) if src_jitter else 0)
    src = (cx, cy, min(sponge_width + 10, n - 1))
    xs = range(n // 4, 3 * n // 4, 2)
    rec = np.array([(ix, iy, min(sponge_width + 5, n - 1)) for iy in xs for ix in xs], dtype=np.int32)
    return Shot(ndim=3, shape=shape, h=h, dt=dt, nt=nt, vel=vel, src=src,
                wavelet=ricker(nt, dt, f), receivers=rec, sponge_width=sponge_width,
                name=f"3d-serve-{n}-{nt}-shot{i}")


def batched_3d_shots(nshots: int = 24, nt: int = 300, seed: int = 6):
    """The batched 3D workload: nshots cubes drawn from {128, ..., 256} (seed), each of
    the serving mix (layered plus random velocity, one model per cube size, sponge 20,
    the source position drawn per shot), nt steps each."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.array([128, 160, 192, 224, 256]), nshots)
    vels = {int(n): serving_3d_velocity(int(n), 5000 + int(n)) for n in set(sizes.tolist())}
    return [serving_3d_shot(i, int(n), nt, vel=vels[int(n)]) for i, n in enumerate(sizes)]


def adjoint_3d(n: int = 256, nt: int = 1500, nshots: int = 8, seed: int = 5, sponge_width: int = 20):
    """The adjoint workload: smoothed random velocity in [1500, 4000] (GRF, 200 m),
    nshots surface shots at seeded positions, and the true model with a +5 %
    Gaussian anomaly (std 150 m) at the centre.  Returns (shots, v_true)."""
    shape = (n, n, n)
    vel = grf_velocity(shape, corr_cells=20.0, vmin=1500.0, vmax=4000.0, seed=seed)
    h, f = 10.0, 10.0
    dt = courant_dt(h, 4000.0 * 1.05)
    rng = np.random.default_rng(seed)
    idx = np.indices(shape, dtype=np.float64)
    r2 = sum((idx[i] - (n - 1) / 2.0) ** 2 for i in range(3)) * h * h
    v_true = (vel.astype(np.float64) * (1.0 + 0.05 * np.exp(-r2 / (2 * 150.0 ** 2)))).astype(np.float32)
    xs = range(n // 8, n - n // 8, 4)
    rec = np.array([(ix, iy, sponge_width + 5) for iy in xs for ix in xs], dtype=np.int32)
    shots = []
    for i in range(nshots):
        sx, sy = (int(q) for q in rng.integers(n // 4, 3 * n // 4, 2))
        shots.append(Shot(ndim=3, shape=shape, h=h, dt=dt, nt=nt, vel=vel, src=(sx, sy, sponge_width + 8),
                          wavelet=ricker(nt, dt, f), receivers=rec, sponge_width=sponge_width,
                          name=f"3d-adjoint-{n}-{nt}-shot{i}"))
    return shots, v_true
