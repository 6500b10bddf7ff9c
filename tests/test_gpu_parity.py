"""GPU path vs the FP64 oracle, through the C ABI (needs a CUDA device).

The procedure is the paper's generic test (section 6): inputs are built on the
host, copied in, the routine runs, outputs are copied back and compared on the
host.  Floating-point results must match the oracle within a relative L2
error of 1e-4 (wavefield and traces); integer maps (source and receiver
indices, sponge band extents) must match exactly.
"""
import os
import warnings

import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

TOL = 1e-4


class MeasuredErrors(UserWarning):
    """The measured errors of a full-size comparison, reported in the test summary."""


def gpu_run(fd, shot, nt, P0=None, Pold0=None):
    with fd.Model.from_shot(shot) as m:
        if P0 is None:
            m.run_shot(nt)
        else:
            fd.fd_set_trace_buffer(m.handle, None, nt)
            fd.fd_set_wavefield(m.handle, P0, Pold0, 0)
            m.step(nt)
        tr = m.traces(nt)
        P, Pold = m.wavefield(with_old=True)
    return P, Pold, tr


def oracle_run(oracle, shot, nt, P0=None, Pold0=None):
    return oracle.run(shot.ndim, shot.shape, shot.h, shot.dt, shot.vel, sponge_width=shot.sponge_width,
                      sponge_R=shot.sponge_R, src=shot.src, wavelet=shot.wavelet, receivers=shot.receivers,
                      P=P0, Pold=Pold0, nsteps=nt)


def assert_parity(gpu, ref, what):
    P, Pold, tr = gpu
    Pr, Poldr, trr = ref
    assert np.all(np.isfinite(P)) and np.all(np.isfinite(tr))
    e_p = pl.rel_l2(P, Pr)
    e_o = pl.rel_l2(Pold, Poldr)
    e_t = pl.rel_l2(tr, trr)
    assert e_p <= TOL and e_o <= TOL and e_t <= TOL, (what, e_p, e_o, e_t)
    return e_p, e_t


# ------------------------------------------------------------------ workloads

def test_parity_2d_workload(fdlib, oracle):
    """256 x 256, 500 steps, 15 Hz Ricker, 64 receivers, rigid boundaries."""
    shot = wl.parity_2d()
    assert_parity(gpu_run(fdlib, shot, shot.nt), oracle_run(oracle, shot, shot.nt), "2d")


def test_parity_2d_ragged_sponge(fdlib, oracle):
    """Ragged 53 x 77 grid (tiles 64 x 16 leave tails), random velocity, sponge 6."""
    shape = (53, 77)
    vel = wl.grf_velocity(shape, corr_cells=6.0, seed=21)
    dt = wl.courant_dt(10.0, float(vel.max()))
    nt = 400
    rng = np.random.default_rng(22)
    rec = np.array([(ix, 0, 11) for ix in range(0, 77, 3)] +
                   [(int(rng.integers(0, 77)), 0, int(rng.integers(0, 53))) for _ in range(20)], np.int32)
    shot = wl.Shot(2, shape, 10.0, dt, nt, vel, (30, 0, 20), wl.ricker(nt, dt, 20.0), rec, sponge_width=6)
    assert_parity(gpu_run(fdlib, shot, nt), oracle_run(oracle, shot, nt), "2d ragged")


def test_parity_3d_ragged_sponge(fdlib, oracle):
    """45 x 38 x 70 grid: several (x, y) tiles with tails, two z chunks, sponge 8."""
    shot = wl.roofline_3d(shape=(45, 38, 70), nt=300, sponge_width=8)
    assert_parity(gpu_run(fdlib, shot, shot.nt), oracle_run(oracle, shot, shot.nt), "3d ragged")


def test_parity_3d_layered_96(fdlib, oracle):
    """The layered 3D workload at 96^3 with a 20-point sponge, 400 steps."""
    shot = wl.roofline_3d(n=96, nt=400, sponge_width=20)
    assert_parity(gpu_run(fdlib, shot, shot.nt), oracle_run(oracle, shot, shot.nt), "3d 96")


def test_parity_3d_full_size_from_random_state(fdlib, oracle):
    """512^3 layered workload (the benchmark's launch configuration), random initial
    levels so every point, face and sponge band is active, 3 steps with the source on."""
    shot = wl.roofline_3d(n=512, nt=3)
    P0, Pm1 = wl.random_state(shot.shape, seed=31)
    gpu = gpu_run(fdlib, shot, 3, P0, Pm1)
    ref = oracle_run(oracle, shot, 3, P0, Pm1)
    assert_parity(gpu, ref, "3d 512 state")
    # pointwise: FP32 rounding of a few steps only
    err = np.max(np.abs(gpu[0] - ref[0])) / np.max(np.abs(ref[0]))
    assert err < 1e-5, err


def test_full_size_reciprocity(fdlib):
    """512^3, 1000 steps, sponge on: v_s^2 P_(s->r) = v_r^2 P_(r->s) on the GPU."""
    shot = wl.roofline_3d(n=512, nt=1000)
    s = shot.src
    r = (shot.nx // 2 + 60, shot.ny // 2 - 40, 25 + 60)
    v = shot.vel
    vs, vr = float(v[s[2], s[1], s[0]]), float(v[r[2], r[1], r[0]])
    out = []
    for a, b in ((s, r), (r, s)):
        sh = wl.Shot(3, shot.shape, shot.h, shot.dt, shot.nt, v, a, shot.wavelet,
                     np.array([b], np.int32), sponge_width=shot.sponge_width)
        with fdlib.Model.from_shot(sh) as m:
            m.run_shot(shot.nt)
            out.append(m.traces(shot.nt)[:, 0].astype(np.float64))
    lhs, rhs = vs * vs * out[0], vr * vr * out[1]
    assert np.max(np.abs(lhs)) > 0
    assert pl.rel_l2(lhs, rhs) < TOL


# ------------------------------------------------------------------ exact maps

def test_index_maps_are_exact(fdlib, oracle):
    shot = wl.roofline_3d(shape=(40, 36, 50), nt=4, sponge_width=7)
    with fdlib.Model.from_shot(shot) as m:
        nz, ny, nx = shot.shape
        sx, sy, sz = shot.src
        assert fdlib.fd_get_source_index(m.handle) == (sz * ny + sy) * nx + sx
        rec = shot.receivers.astype(np.int64)
        want = (rec[:, 2] * ny + rec[:, 1]) * nx + rec[:, 0]
        np.testing.assert_array_equal(fdlib.fd_get_receiver_indices(m.handle, len(rec)), want)
        emax = oracle.sponge_eta_max(float(shot.vel.max()), 7, shot.h, shot.sponge_R)
        for axis, n in ((0, nx), (1, ny), (2, nz)):
            got = fdlib.fd_get_damping_profile(m.handle, axis, n)
            ref = shot.dt * oracle.sponge_profile(n, 7, emax)
            np.testing.assert_array_equal(got != 0, ref != 0)          # band extents, exactly
            np.testing.assert_allclose(got, ref, rtol=2e-7, atol=0)    # values, FP32 rounding


def test_2d_has_no_y_damping(fdlib):
    shot = wl.parity_2d(nt=2)
    shot.sponge_width = 5
    with fdlib.Model.from_shot(shot) as m:
        assert np.all(fdlib.fd_get_damping_profile(m.handle, 1, 1) == 0)
        assert np.count_nonzero(fdlib.fd_get_damping_profile(m.handle, 0, 256)) == 10


# ------------------------------------------------------------------ edge cases

def test_zero_steps_and_empty_receivers(fdlib):
    shot = wl.parity_2d(nt=5)
    with fdlib.Model.from_shot(shot) as m:
        m.run_shot(0)
        assert m.traces(0).shape == (0, 64)
        assert np.all(m.wavefield() == 0)
        m.set_receivers(np.zeros((0, 3), np.int32))
        m.run_shot(5)
        assert m.traces(5).shape == (5, 0)
        assert np.any(m.wavefield() != 0)


def test_split_steps_equal_one_call_bitwise(fdlib):
    shot = wl.roofline_3d(shape=(33, 20, 40), nt=12, sponge_width=4)
    with fdlib.Model.from_shot(shot) as m:
        m.run_shot(12)
        P1, tr1 = m.wavefield(), m.traces(12)
        fdlib.fd_reset(m.handle)
        fdlib.fd_set_trace_buffer(m.handle, None, 12)
        for n in (3, 0, 5, 4):
            m.step(n)
        assert fdlib.fd_get_step(m.handle) == 12
        np.testing.assert_array_equal(m.wavefield(), P1)
        np.testing.assert_array_equal(m.traces(12), tr1)


def test_deterministic_bitwise(fdlib):
    shot = wl.roofline_3d(n=64, nt=30)
    a = gpu_run(fdlib, shot, 30)
    b = gpu_run(fdlib, shot, 30)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (1, 9), (9, 1), (2, 3, 1), (1, 1, 1), (5, 3, 4)])
def test_tiny_grids(fdlib, oracle, shape):
    ndim = len(shape)
    rng = np.random.default_rng(41)
    vel = rng.uniform(1500, 2500, shape).astype(np.float32)
    dt = 0.3 * 10.0 / float(vel.max())
    nt = 25
    pts = [(0, 0, 0), (shape[-1] - 1, 0 if ndim == 2 else shape[1] - 1, shape[0] - 1)]
    rec = np.array(pts, np.int32)
    shot = wl.Shot(ndim, shape, 10.0, dt, nt, vel, pts[-1], wl.ricker(nt, dt, 30.0), rec)
    P0, Pm1 = wl.random_state(shape, seed=42)
    assert_parity(gpu_run(fdlib, shot, nt, P0, Pm1), oracle_run(oracle, shot, nt, P0, Pm1), f"tiny {shape}")


def test_source_and_receivers_at_corners(fdlib, oracle):
    shape = (30, 18, 26)
    vel = wl.layered_velocity(shape, seed=5)
    dt = wl.courant_dt(10.0, float(vel.max()))
    nt = 60
    nz, ny, nx = shape
    corners = [(x, y, z) for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    shot = wl.Shot(3, shape, 10.0, dt, nt, vel, (0, 0, 0), wl.ricker(nt, dt, 40.0),
                   np.array(corners, np.int32), sponge_width=5)
    assert_parity(gpu_run(fdlib, shot, nt), oracle_run(oracle, shot, nt), "corners")


# ------------------------------------------------------------------ errors

def test_out_of_range_points_are_erange(fdlib):
    shot = wl.roofline_3d(shape=(20, 20, 20), nt=5, sponge_width=0)
    with fdlib.Model.from_shot(shot) as m:
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_set_source(m.handle, 20, 0, 0, shot.wavelet)
        assert e.value.status == fdlib.FD_ERANGE
        with pytest.raises(fdlib.FDError) as e:
            m.set_receivers(np.array([(0, 0, 0), (0, -1, 3)], np.int32))
        assert e.value.status == fdlib.FD_ERANGE
        # the rejected calls changed nothing
        assert fdlib.fd_get_source_index(m.handle) == (shot.src[2] * 20 + shot.src[1]) * 20 + shot.src[0]
        np.testing.assert_array_equal(fdlib.fd_get_receiver_indices(m.handle, len(shot.receivers)),
                                      (shot.receivers[:, 2].astype(np.int64) * 20 + shot.receivers[:, 1]) * 20
                                      + shot.receivers[:, 0])


def test_rejected_velocity_leaves_model_unchanged(fdlib):
    import torch
    shot = wl.roofline_3d(shape=(24, 20, 36), nt=20, sponge_width=4)
    with fdlib.Model.from_shot(shot) as m:
        m.run_shot(20)
        P1 = m.wavefield()
        fast = np.full(shot.vel.size, 1e5, np.float32)
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_set_velocity(m.handle, fast)
        assert e.value.status == fdlib.FD_ECFL
        bad = torch.full((shot.vel.size,), 2000.0, device="cuda")
        bad[17] = float("nan")
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_set_velocity_dev(m.handle, bad)
        assert e.value.status == fdlib.FD_EINVAL
        m.run_shot(20)
        np.testing.assert_array_equal(m.wavefield(), P1)


def test_device_inputs_match_host_inputs(fdlib):
    import torch
    shot = wl.roofline_3d(shape=(24, 20, 36), nt=15, sponge_width=4)
    a = gpu_run(fdlib, shot, 15)
    v_dev = torch.from_numpy(shot.vel.ravel()).cuda()
    traces = torch.zeros((15, len(shot.receivers)), device="cuda")
    with fdlib.Model(3, shot.shape, shot.h, shot.dt, v_dev, shot.sponge_width) as m:
        m.set_source(shot.src, shot.wavelet)
        m.set_receivers(shot.receivers)
        m.run_shot(15, traces)
        fdlib.fd_synchronize(m.handle)
        np.testing.assert_array_equal(m.wavefield(), a[0])
    np.testing.assert_array_equal(traces.cpu().numpy(), a[2])


def test_async_trace_gather(fdlib):
    """fd_gather_traces_async enqueues the same copy as fd_gather_traces without
    waiting; after fd_synchronize the pinned buffer holds the same traces."""
    import torch
    shot = wl.roofline_3d(shape=(33, 20, 40), nt=12, sponge_width=4)
    with fdlib.Model.from_shot(shot) as m:
        m.run_shot(shot.nt)
        want = m.traces(shot.nt)
        m.run_shot(shot.nt)
        buf = torch.full((shot.nt, len(shot.receivers)), float("nan")).pin_memory()
        fdlib.fd_gather_traces_async_ptr(m.handle, buf.data_ptr(), buf.numel())
        fdlib.fd_synchronize(m.handle)
        np.testing.assert_array_equal(buf.numpy(), want)
        with pytest.raises(fdlib.FDError):
            fdlib.fd_gather_traces_async_ptr(m.handle, buf.data_ptr(), buf.numel() - 1)


def _sample_points(shape, bz, rng, nrandom=200):
    """Tile and chunk edges, faces, corners and random points of a grid."""
    axes = []
    for ax, n in enumerate(shape):
        cand = {0, 1, 3, 4, 5, n // 2, n - 5, n - 4, n - 2, n - 1}
        if ax == len(shape) - 1:
            cand |= {31, 32, 33, 63, 64, 65}            # x tile edges (32 in 3D, 64 in 2D)
        elif ax == 0 and len(shape) == 3:
            cand |= {bz - 1, bz, bz + 1}                 # z chunk edge
        else:
            cand |= {15, 16, 17, 31, 32, 33}             # y / 2D z tile edges
        axes.append(sorted(c for c in cand if 0 <= c < n))
    grid = np.array(np.meshgrid(*axes, indexing="ij")).reshape(len(shape), -1).T
    pick = grid[rng.choice(len(grid), size=min(len(grid), 400), replace=False)]
    rnd = np.stack([rng.integers(0, n, nrandom) for n in shape], axis=1)
    return np.concatenate([pick, rnd])


@pytest.mark.parametrize("shape", [(520, 2050, 2046), (40000, 56000)])
def test_parity_beyond_2pow31_points_sampled(fdlib, oracle, shape):
    """Grids of more than 2^31 points, so every index path needs 64 bits: one step
    from a random state, checked at sampled points (tile and chunk edges, faces,
    corners, random points).  Each reference value is the oracle's step of the
    point's radius-4 neighbourhood cut from the same inputs; no sponge, so the cut
    sees the same coefficients, and where it meets a grid face the oracle's zero
    halo is the grid's own."""
    import torch
    ndim = len(shape)
    assert int(np.prod(shape)) > 2 ** 31
    h = 10.0
    dt = 0.4 * h / 2500.0
    vel, P0, Pm1 = wl.device_random_fields(shape, seed=77)
    out = torch.empty_like(P0)
    with fdlib.Model(ndim, shape, h, dt, vel) as m:
        fdlib.fd_set_wavefield_dev(m.handle, P0, Pm1, 0)
        fdlib.fd_step(m.handle, 1)
        fdlib.fd_get_wavefield_dev(m.handle, out)
        torch.cuda.synchronize()
    pts = _sample_points(shape, 512, np.random.default_rng(5))
    idx = tuple(torch.from_numpy(pts[:, a]).cuda() for a in range(ndim))
    got = out[idx].double().cpu().numpy()
    ref = np.empty(len(pts))
    for i, p in enumerate(pts):
        lo = [max(0, c - 4) for c in p]
        hi = [min(n, c + 5) for c, n in zip(p, shape)]
        cut = tuple(slice(a, b) for a, b in zip(lo, hi))
        Pn, _, _ = oracle.run(ndim, tuple(b - a for a, b in zip(lo, hi)), h, dt, vel[cut].cpu().numpy(),
                              P=P0[cut].cpu().numpy(), Pold=Pm1[cut].cpu().numpy(), nsteps=1)
        ref[i] = Pn[tuple(c - a for c, a in zip(p, lo))]
    del vel, P0, Pm1, out
    torch.cuda.empty_cache()
    err = np.abs(got - ref) / np.max(np.abs(ref))
    assert err.max() < 1e-5, (err.max(), pts[np.argmax(err)])


@pytest.mark.parametrize("shape,path", [(s, p) for s in [(45, 38, 70), (53, 77)]
                                        for p in ("fused", "unfused", "lp", "batch") if len(s) == 2 or p != "batch"])
def test_padding_canaries_never_reach_a_result(fdlib, oracle, shape, path):
    """NaN in every row's padding (columns nx .. px-1 of P, Pold, w and the unfused
    derivative fields) must never reach a result: every step path reads and writes
    only the nx valid columns.  Checked against the oracle from a random state."""
    import torch
    ndim = len(shape)
    nt = 12
    rng = np.random.default_rng(8)
    vel = rng.uniform(1500, 2500, shape).astype(np.float32)
    dt = 0.4 * 10.0 / 2500.0
    src = (shape[-1] // 3, shape[1] // 2 if ndim == 3 else 0, shape[0] // 2)
    rec = np.array([(x, src[1], 5) for x in range(0, shape[-1], 5)], np.int32)
    shot = wl.Shot(ndim, shape, 10.0, dt, nt, vel, src, wl.ricker(nt, dt, 30.0), rec, sponge_width=5)
    P0, Pm1 = wl.random_state(shape, seed=81)
    lp = torch.zeros(shape, device="cuda")
    with fdlib.Model.from_shot(shot) as m:
        fdlib.fd_set_trace_buffer(m.handle, None, nt)
        fdlib.fd_set_wavefield(m.handle, P0, Pm1, 0)
        if path == "unfused":
            fdlib.fd_routine(m.handle, fdlib.FD_ROUTINE_PXX)     # allocate the derivative fields
        fdlib.fd_debug_poison_padding(m.handle)
        if path == "fused":
            fdlib.fd_step(m.handle, nt)
        elif path == "unfused":
            fdlib.fd_step_unfused(m.handle, nt)
        elif path == "batch":
            with fdlib.Batch([m]) as b:
                b.step(nt)
        else:
            fdlib.fd_step_lp(m.handle, lp)
            fdlib.fd_step(m.handle, nt - 1)
        (P, Pold), tr = m.wavefield(with_old=True), m.traces(nt)
    assert np.isfinite(P).all() and np.isfinite(Pold).all() and np.isfinite(tr).all()
    rP, rPold, rtr = oracle.run(ndim, shape, 10.0, dt, vel, sponge_width=5, src=src, wavelet=shot.wavelet,
                                receivers=rec, P=P0, Pold=Pm1, nsteps=nt)
    assert max(pl.rel_l2(P, rP), pl.rel_l2(Pold, rPold), pl.rel_l2(tr, rtr)) <= 1e-4
    if path == "lp":
        got = lp.cpu().numpy()
        assert np.isfinite(got).all() and pl.rel_l2(got, oracle.stencil_sum(P0)) <= 1e-6


def test_parity_3d_long_run_2000_steps(fdlib, oracle):
    """FP32 drift over a long run: 64^3 layered model with sponge, source and
    receivers, 2000 steps (twice the benchmark's shot length) against the FP64
    oracle, rel L2 <= 1e-4 (the D_k form of the stencil keeps the phase error of
    FP32 rounding from growing into a spurious mass term)."""
    shot = wl.roofline_3d(n=64, nt=2000, sponge_width=10)
    assert_parity(gpu_run(fdlib, shot, shot.nt), oracle_run(oracle, shot, shot.nt), "3d 64 long run")


@pytest.mark.parametrize("shape", [(64, 96), (40, 44, 52)])
@pytest.mark.parametrize("sponge", [0, 6])
def test_gpu_discrete_energy(fdlib, shape, sponge):
    """An oracle-free property of the GPU step: with no source, the discrete energy
    E^(n+1/2) = sum (Pn - P)^2 / w - sum Pn L'P (FP64 from the FP32 levels) is
    constant to FP32 rounding over 2000 steps without a sponge, and never grows
    with one.  It holds only for a symmetric stencil under the zero halo."""
    ndim = len(shape)
    h = 10.0
    v = wl.grf_velocity(shape, corr_cells=4.0, vmin=1500.0, vmax=3000.0, seed=12)
    dt = 0.4 * h / float(v.max())
    f = wl.random_field(shape, 3.0, 13)
    P0 = (f / f.std()).astype(np.float32)
    Pm1 = (np.roll(f, 1, axis=-1) / f.std()).astype(np.float32)
    c = pl.fornberg_coefficients(4)
    w = (dt * v.astype(np.float64) / h) ** 2
    E = []
    with fdlib.Model(ndim, shape, h, dt, v, sponge) as m:
        fdlib.fd_set_wavefield(m.handle, P0, Pm1, 0)
        for _ in range(20):
            fdlib.fd_step(m.handle, 100)
            P, Pold = m.wavefield(with_old=True)
            E.append(pl.energy(Pold.astype(np.float64), P.astype(np.float64), w, c))
    E = np.array(E)
    assert np.all(E > 0)
    if sponge == 0:
        assert np.max(np.abs(E - E[0])) / E[0] < 1e-4, E
    else:
        assert np.all(np.diff(E) <= 1e-6 * E[0]), E
        assert E[-1] < 0.5 * E[0]


@pytest.mark.parametrize("stage", [0, 6])
def test_step_kernel_wait_times_out_and_context_survives(fdlib, oracle, stage):
    """A P stage that never arrives (the test hook keeps the first CTA from issuing
    it: an initial stage, or a refill) runs that CTA's bounded waits out: the next
    synchronisation reports FD_ETIMEOUT within seconds, and a clean run on the same
    model then matches the oracle.  Nothing faults, traps or hangs."""
    import time
    shot = wl.roofline_3d(shape=(40, 36, 70), nt=30, sponge_width=6)
    with fdlib.Model.from_shot(shot) as m:
        fdlib.fd_debug_stall_stage(m.handle, stage)
        t0 = time.perf_counter()
        fdlib.fd_step(m.handle, 1)
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_synchronize(m.handle)
        assert e.value.status == -7                      # FD_ETIMEOUT
        assert time.perf_counter() - t0 < 30
        fdlib.fd_debug_stall_stage(m.handle, -1)
        fdlib.fd_reset(m.handle)
        fdlib.fd_set_trace_buffer(m.handle, None, shot.nt)
        fdlib.fd_step(m.handle, shot.nt)
        tr = m.traces(shot.nt)
        P, Pold = m.wavefield(with_old=True)
    assert_parity((P, Pold, tr), oracle_run(oracle, shot, shot.nt), f"after a timeout at stage {stage}")


# ------------------------------------------------------------ full benchmark shot

GOLDEN_ROOFLINE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                               "roofline_3d_512_1000steps_oracle.npz")


def test_parity_3d_roofline_full_run(fdlib):
    """The benchmark's shot (512^3 layered, sponge 20, 10 Hz source, 65 536 receivers)
    over all 1000 steps through fd_run_shot, against the FP64 oracle's run of the
    same inputs (section 7, Eq. 1).

    The oracle's outputs are stored as a digest written by
    tests/golden/make_roofline_3d_digest.py, which calls only the oracle.  Checks:
    element by element on the final P over the vertical plane through the source
    and on the traces of the receiver row through the source (rel L2 <= 1e-4),
    and over the WHOLE final P, Pold and trace array through their CountSketches,
    whose difference estimates the full rel L2 to about 1 % of itself (bar 1e-4).
    """
    import digest
    ref = np.load(GOLDEN_ROOFLINE)
    shot = wl.roofline_3d(n=512, nt=1000)
    assert str(ref["name"]) == shot.name and tuple(ref["shape"]) == shot.shape
    P, Pold, tr = gpu_run(fdlib, shot, shot.nt)
    assert np.all(np.isfinite(P)) and np.all(np.isfinite(Pold)) and np.all(np.isfinite(tr))
    iy = int(ref["plane_iy"])
    row = ref["row_receivers"]
    e_plane = pl.rel_l2(P[:, iy, :], ref["plane_P"])
    e_row = pl.rel_l2(tr[:, row], ref["row_traces"])
    k, seed = int(ref["sketch_k"]), int(ref["sketch_seed"])
    (nP, nO), (yP, yO) = digest.sketch([P, Pold], k, seed)
    (nT,), (yT,) = digest.sketch([tr], k, seed)
    e_P = digest.sketch_rel_l2(yP, ref["sketch_P"], float(ref["norm_P"]))
    e_O = digest.sketch_rel_l2(yO, ref["sketch_Pold"], float(ref["norm_Pold"]))
    e_T = digest.sketch_rel_l2(yT, ref["sketch_traces"], float(ref["norm_traces"]))
    msg = (f"512^3 x 1000 vs oracle: plane {e_plane:.2e}, receiver row {e_row:.2e}; "
           f"whole P {e_P:.2e}, Pold {e_O:.2e}, traces {e_T:.2e} (sketch estimates); "
           f"norms {nP / float(ref['norm_P']) - 1:+.1e} {nO / float(ref['norm_Pold']) - 1:+.1e} "
           f"{nT / float(ref['norm_traces']) - 1:+.1e}")
    print(msg)
    # also as a warning, so that the measured errors show in a quiet (-q) run's summary
    warnings.warn(MeasuredErrors(msg))
    assert max(e_plane, e_row, e_P, e_O, e_T) <= TOL, (e_plane, e_row, e_P, e_O, e_T)
    for got, key in ((nP, "norm_P"), (nO, "norm_Pold"), (nT, "norm_traces")):
        assert abs(got / float(ref[key]) - 1.0) <= TOL, key


def test_parity_2d_large_grid_stacked_tiles(fdlib, oracle):
    """A 2D grid large enough for the step kernel's columns of 8 stacked tiles
    (8150 x 4100: ragged in x and in the last column's tile count), from a random
    state with sponge, source and receivers: against the oracle (rel L2 <= 1e-4),
    and bitwise against the same steps through the wide batch schedule with one
    tile per CTA (the same per-tile arithmetic)."""
    shape = (8150, 4100)
    rng = np.random.default_rng(61)
    vel = rng.uniform(1500.0, 3000.0, shape).astype(np.float32)
    dt = wl.courant_dt(10.0, 3000.0)
    nt = 4
    rec = np.array([(int(rng.integers(0, 4100)), 0, int(rng.integers(0, 8150))) for _ in range(300)], np.int32)
    shot = wl.Shot(2, shape, 10.0, dt, nt, vel, (2049, 0, 4001), wl.ricker(nt, dt, 15.0, t0=0.0), rec,
                   sponge_width=10)
    P0, Pm1 = wl.random_state(shape, seed=62)
    out = []
    for batched in (False, True):
        with fdlib.Model.from_shot(shot) as m:
            fdlib.fd_set_trace_buffer(m.handle, None, nt)
            fdlib.fd_set_wavefield(m.handle, P0, Pm1, 0)
            if batched:
                with fdlib.Batch([m]) as b:
                    b.set_tuning(tile=3, steps_per_launch=2000, ctas_per_sm=0, group_mb=0)
                    b.step(nt)
            else:
                m.step(nt)
            out.append((*m.wavefield(with_old=True), m.traces(nt)))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    ref = oracle.run(2, shape, shot.h, dt, vel, sponge_width=10, src=shot.src, wavelet=shot.wavelet,
                     receivers=rec, P=P0, Pold=Pm1, nsteps=nt)
    assert max(pl.rel_l2(g, r) for g, r in zip(out[0], ref)) <= TOL
