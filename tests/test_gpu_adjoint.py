"""Reverse-time adjoint on the GPU: gradient w.r.t. squared slowness (needs a CUDA device).

Checked against the FP64 oracle's discrete-adjoint gradient (which is itself
pinned to finite differences), against finite differences of the GPU misfit,
and for independence from the checkpoint interval.
"""
import numpy as np
import pytest

import pinlib as pl
import workloads as wl
from conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def case(ndim, nt=120, seed=3):
    if ndim == 2:
        shape = (60, 72)
        src = (36, 0, 10)
        rec = np.array([(x, 0, 8) for x in range(6, 66, 3)], np.int32)
    else:
        shape = (36, 32, 40)
        src = (20, 16, 9)
        rec = np.array([(x, y, 7) for y in range(6, 26, 4) for x in range(6, 34, 4)], np.int32)
    v = wl.grf_velocity(shape, corr_cells=4.0, vmin=1800.0, vmax=3000.0, seed=seed)
    h = 10.0
    dt = 0.35 * h / 3200.0
    idx = np.indices(shape)
    blob = np.exp(-sum((idx[i] - shape[i] / 2) ** 2 for i in range(ndim)) / (2 * 5.0 ** 2))
    vt = (v * (1.0 + 0.2 * blob)).astype(np.float32)   # a strong anomaly keeps the residual well above FP32 rounding
    shot = wl.Shot(ndim, shape, h, dt, nt, v, src, wl.ricker(nt, dt, 30.0), rec, sponge_width=6)
    return shot, vt


def observed(fd, shot, vt, vmax):
    import torch
    s2 = wl.Shot(shot.ndim, shot.shape, shot.h, shot.dt, shot.nt, vt, shot.src, shot.wavelet, shot.receivers,
                 sponge_width=shot.sponge_width)
    with fd.Model.from_shot(s2) as m:
        fd.fd_set_sponge_vmax(m.handle, vmax)
        m.run_shot(shot.nt)
        return torch.from_numpy(m.traces(shot.nt)).cuda()


def velocity_of(m):
    """The FP32 velocity the library derives from squared slowness m (FP64, one rounding)."""
    return (1.0 / np.sqrt(m.cpu().numpy().astype(np.float64))).astype(np.float32)


def gpu_and_oracle(fd, oracle, shot, observed_np, vmax=3200.0, K=25):
    import torch
    from paper_2311_05038_b300 import adjoint
    geo = adjoint.Geometry.from_shot(shot, checkpoint_every=K, sponge_vmax=vmax)
    m = torch.from_numpy((1.0 / shot.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    J, g = adjoint.misfit_and_gradient(m, geo, torch.from_numpy(observed_np.astype(np.float32)).cuda())
    Jr, gr, _ = oracle.misfit_gradient(shot.ndim, shot.shape, shot.h, shot.dt, velocity_of(m),
                                       sponge_width=shot.sponge_width, src=shot.src, wavelet=shot.wavelet,
                                       receivers=shot.receivers, nsteps=shot.nt, observed=observed_np,
                                       sponge_vmax=vmax)
    return J, g.cpu().numpy(), Jr, gr


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_matches_oracle_without_data(fdlib, oracle, ndim):
    """J = 1/2 |d|^2: no residual cancellation, so FP32 rounding stays at its own size."""
    shot, _ = case(ndim)
    zero = np.zeros((shot.nt, len(shot.receivers)))
    J, g, Jr, gr = gpu_and_oracle(fdlib, oracle, shot, zero)
    assert J == pytest.approx(Jr, rel=1e-5)
    assert pl.rel_l2(g, gr) <= 1e-4


@pytest.mark.parametrize("ndim,tol", [(3, 1e-3), (2, 5e-3)])
def test_gradient_matches_oracle_for_a_misfit(fdlib, oracle, ndim, tol):
    """Observed data from a model with a 20 % anomaly.  The residual d - d_obs is a
    difference of two FP32 trace sets, so the traces' rounding enters the gradient
    amplified by |d| / |r|; in this 2D geometry (weak reflection back to the
    receivers) that puts the FP32 gradient about 2e-3 from the FP64 one, in 3D
    about 1e-5."""
    shot, vt = case(ndim)
    dobs = observed(fdlib, shot, vt, 3200.0).cpu().numpy().astype(np.float64)
    J, g, Jr, gr = gpu_and_oracle(fdlib, oracle, shot, dobs)
    print(f"{ndim}D reflection misfit: J {J:.6e} vs {Jr:.6e}, gradient rel L2 {pl.rel_l2(g, gr):.2e}")
    assert J == pytest.approx(Jr, rel=1e-3)
    assert pl.rel_l2(g, gr) <= tol


def test_gradient_matches_oracle_in_transmission_2d(fdlib, oracle):
    """The 2D case with the receivers below the anomaly (transmission): the
    residual is then a large part of the traces, FP32 rounding is not amplified,
    and the gradient matches the FP64 one to 1e-4."""
    shot, vt = case(2)
    shot.receivers = np.array([(x, 0, 50) for x in range(6, 66, 3)], np.int32)
    dobs = observed(fdlib, shot, vt, 3200.0).cpu().numpy().astype(np.float64)
    J, g, Jr, gr = gpu_and_oracle(fdlib, oracle, shot, dobs)
    err = pl.rel_l2(g, gr)
    print(f"2D transmission misfit: J {J:.6e} vs {Jr:.6e}, gradient rel L2 {err:.2e}")
    assert J == pytest.approx(Jr, rel=1e-4)
    assert err <= 1e-4


def test_gradient_matches_finite_differences(fdlib):
    import torch
    from paper_2311_05038_b300 import adjoint
    shot, vt = case(3, nt=120, seed=4)
    vmax = 3200.0
    dobs = observed(fdlib, shot, vt, vmax)
    geo = adjoint.Geometry.from_shot(shot, checkpoint_every=40, sponge_vmax=vmax)
    m = torch.from_numpy((1.0 / shot.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    J, g = adjoint.misfit_and_gradient(m, geo, dobs)
    for trial in range(2):
        dm = torch.from_numpy((wl.random_field(shot.shape, 3.0, 200 + trial) * 0.02).astype(np.float32)).cuda() * m
        eps = 0.05
        Jp, _ = adjoint.misfit_and_gradient(m + eps * dm, geo, dobs)
        Jm, _ = adjoint.misfit_and_gradient(m - eps * dm, geo, dobs)
        fdv = (Jp - Jm) / (2 * eps)
        an = float((g.double() * dm.double()).sum())
        assert abs(fdv - an) <= 1e-2 * abs(an), (fdv, an)


def test_gradient_independent_of_checkpoint_interval(fdlib):
    import torch
    from paper_2311_05038_b300 import adjoint
    shot, vt = case(2, nt=90, seed=5)
    dobs = observed(fdlib, shot, vt, 3200.0)
    m = torch.from_numpy((1.0 / shot.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    grads = []
    for K in (1, 13, 90):
        geo = adjoint.Geometry.from_shot(shot, checkpoint_every=K, sponge_vmax=3200.0)
        grads.append(adjoint.misfit_and_gradient(m, geo, dobs)[1].cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])
    np.testing.assert_array_equal(grads[0], grads[2])


def _random_shot(shape, seed):
    rng = np.random.default_rng(seed)
    vel = rng.uniform(1500, 2500, shape).astype(np.float32)
    ndim = len(shape)
    dt = 0.4 * 10.0 / 2500.0
    src = tuple(int(rng.integers(0, n)) for n in reversed(shape)) if ndim == 3 else \
        (int(rng.integers(0, shape[1])), 0, int(rng.integers(0, shape[0])))
    nt = 4
    return wl.Shot(ndim, shape, 10.0, dt, nt, vel, src, wl.ricker(nt, dt, 30.0), np.zeros((0, 3), np.int32),
                   sponge_width=3)


@pytest.mark.parametrize("shape", [(36, 32, 40), (21, 17, 29), (45, 38, 70), (60, 72), (33, 45)])
def test_step_lp_writes_the_stencil_sum(fdlib, oracle, shape):
    """fd_step_lp advances exactly as fd_step (bitwise) and writes L'P of the level it
    consumed at every point, dense; nx = 29 and 45 take the unaligned store path, and
    nz = 21, 33, 45 leave an odd plane count in a 3D chunk."""
    import torch
    shot = _random_shot(shape, seed=sum(shape))
    P0, Pm1 = wl.random_state(shape, seed=len(shape) * 100 + shape[-1])
    with fdlib.Model.from_shot(shot) as a, fdlib.Model.from_shot(shot) as b:
        for m in (a, b):
            fdlib.fd_set_wavefield(m.handle, P0, Pm1, 0)
        lp = torch.full(shape, float("nan"), device="cuda")
        fdlib.fd_step_lp(a.handle, lp)
        fdlib.fd_step(b.handle, 1)
        np.testing.assert_array_equal(a.wavefield(), b.wavefield())
        got = lp.cpu().numpy()
    assert np.isfinite(got).all()
    assert pl.rel_l2(got, oracle.stencil_sum(P0)) <= 1e-6


@pytest.mark.parametrize("shape", [(21, 17, 29), (33, 45)])
def test_imaging_product(fdlib, shape):
    """grad += psi * lp pointwise, psi the adjoint model's current level."""
    import torch
    shot = _random_shot(shape, seed=7)
    psi, lp = wl.random_state(shape, seed=11)
    g0 = np.random.default_rng(12).standard_normal(shape).astype(np.float32)
    with fdlib.Model.from_shot(shot) as adj:
        fdlib.fd_set_wavefield(adj.handle, psi, np.zeros(shape, np.float32), 0)
        grad = torch.from_numpy(g0).cuda()
        fdlib.fd_imaging_product(adj.handle, torch.from_numpy(lp).cuda(), grad)
        got = grad.cpu().numpy()
    want = g0.astype(np.float64) + psi.astype(np.float64) * lp.astype(np.float64)
    assert np.max(np.abs(got - want) / (np.abs(want) + 1e-3)) <= 1e-6


def _segment_case(fdlib, shape, seed):
    shot = _random_shot(shape, seed)
    rng = np.random.default_rng(seed)
    ndim = len(shape)
    rec = np.array([(int(rng.integers(0, shape[-1])), int(rng.integers(0, shape[1])) if ndim == 3 else 0,
                     int(rng.integers(0, shape[0]))) for _ in range(9)], np.int32)
    shot.receivers = rec
    return shot


@pytest.mark.parametrize("shape", [(21, 17, 29), (33, 45)])
def test_adjoint_segment_equals_step_by_step_calls(fdlib, shape):
    """fd_adjoint_segment issues exactly fd_step_lp x (n1-n0), then per k
    fd_step_image and fd_inject_receivers_image: results bitwise equal."""
    import torch
    shot = _segment_case(fdlib, shape, seed=5)
    n0, n1 = 3, 9
    P, Po = wl.random_state(shape, seed=21)
    psi, psio = wl.random_state(shape, seed=22, scale=1e-3)
    g = torch.from_numpy(np.random.default_rng(23).standard_normal((n1, len(shot.receivers))).astype(np.float32)).cuda()
    out = []
    for native in (True, False):
        with fdlib.Model.from_shot(shot) as fwd, fdlib.Model.from_shot(shot) as adj:
            fdlib.fd_set_wavefield(fwd.handle, P, Po, n0)
            fdlib.fd_set_wavefield(adj.handle, psi, psio, 0)
            lp = torch.zeros((n1 - n0,) + shape, device="cuda")
            grad = torch.zeros(shape, device="cuda")
            if native:
                fdlib.fd_adjoint_segment(fwd.handle, adj.handle, n0, n1, lp, g, grad)
            else:
                for j in range(n1 - n0):
                    fdlib.fd_step_lp(fwd.handle, lp[j])
                for k in range(n1, n0, -1):
                    fdlib.fd_step_image(adj.handle, lp[k - 1 - n0], grad)
                    fdlib.fd_inject_receivers_image(adj.handle, g[k - 1], lp[k - 1 - n0], grad)
            torch.cuda.synchronize()
            out.append((lp.cpu().numpy(), grad.cpu().numpy(), adj.wavefield()))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    assert np.abs(out[0][1]).max() > 0


def test_adjoint_segment_argument_checks(fdlib):
    import torch
    shape = (21, 17, 29)
    shot = _segment_case(fdlib, shape, seed=6)
    g = torch.zeros((8, len(shot.receivers)), device="cuda")
    lp = torch.zeros((4,) + shape, device="cuda")
    grad = torch.zeros(shape, device="cuda")
    with fdlib.Model.from_shot(shot) as fwd, fdlib.Model.from_shot(shot) as adj:
        fdlib.fd_step(fwd.handle, 1)                      # forward model at step 1, not 0
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_adjoint_segment(fwd.handle, adj.handle, 0, 4, lp, g, grad)
        assert e.value.status == -8                        # FD_ESTATE
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_adjoint_segment(fwd.handle, adj.handle, 1, 1, lp, g, grad)
        assert e.value.status == -1                        # FD_EINVAL


def test_gradient_full_size_finite_differences(fdlib):
    """The adjoint workload at full size (its 256^3 model, first shot, 1500 steps)
    against central finite differences of the misfit.

    - Zero observed data, J = 1/2 |d|^2, along three smooth random directions of
      2 % rms: agreement within 1e-3 (measured 1e-4 .. 3e-4 at eps = 0.01).
    - The real misfit against data of the +5 % anomaly model, along the anomaly's
      own Gaussian blob, where J is close to quadratic: within 1e-3 (measured
      1.3e-4 at eps = 0.05).

    The real misfit is not differenced along smooth global directions: the
    receivers sit three cells from the source, so such a direction changes the
    direct arrivals by far more than the weak scattered residual, and the FP32
    rounding of those arrivals swamps the misfit's change (two small steps then
    disagree with each other by up to 18 %)."""
    import torch
    from paper_2311_05038_b300 import adjoint
    shots, v_true = wl.adjoint_3d(256, 1500, 1)
    s = shots[0]
    vmax = 4000.0 * 1.05
    geo = adjoint.Geometry.from_shot(s, checkpoint_every=50, sponge_vmax=vmax)
    m = torch.from_numpy((1.0 / s.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()

    def misfit(mm, dobs):
        with torch.no_grad():
            r = (adjoint.Propagate.apply(mm, geo) - dobs).double()
        return 0.5 * float((r * r).sum())

    def check(dobs, dm, eps, tol, what):
        _, g = adjoint.misfit_and_gradient(m, geo, dobs)
        an = float((g.double() * dm.double()).sum())
        fdv = (misfit(m + eps * dm, dobs) - misfit(m - eps * dm, dobs)) / (2 * eps)
        print(f"256^3 finite differences, {what}: relative difference {abs(fdv - an) / abs(an):.2e}")
        assert abs(fdv - an) <= tol * abs(an), (what, fdv, an)

    zero = torch.zeros((s.nt, len(s.receivers)), device="cuda")
    for seed in (300, 301, 302):
        f = wl.random_field(s.shape, 20.0, seed)
        dm = torch.from_numpy((f / f.std() * 0.02).astype(np.float32)).cuda() * m
        check(zero, dm, 0.01, 1e-3, f"zero data, direction {seed}")

    st = wl.Shot(3, s.shape, s.h, s.dt, s.nt, v_true, s.src, s.wavelet, s.receivers, sponge_width=s.sponge_width)
    with fdlib.Model.from_shot(st) as mt:
        fdlib.fd_set_sponge_vmax(mt.handle, vmax)
        mt.run_shot(s.nt)
        dobs = torch.from_numpy(mt.traces(s.nt)).cuda()
    blob = torch.from_numpy((v_true.astype(np.float64) / s.vel - 1.0).astype(np.float32)).cuda()
    check(dobs, -2.0 * blob * m, 0.05, 1e-3, "anomaly data, blob direction")


@pytest.mark.parametrize("shape", [(21, 17, 29), (33, 45), (20, 16, 32)])
def test_fused_imaging_equals_separate_calls(fdlib, shape):
    """fd_step_image is fd_step followed by fd_imaging_product, bitwise (the same FMA
    on the same level); fd_inject_receivers_image adds its share so that the whole
    equals (level + injection) * lp up to one rounding at the receivers."""
    import torch
    shot = _segment_case(fdlib, shape, seed=9)
    P, Po = wl.random_state(shape, seed=31)
    lp = torch.from_numpy(wl.random_state(shape, seed=32)[0]).cuda()
    vals = torch.from_numpy(np.random.default_rng(33).standard_normal(len(shot.receivers)).astype(np.float32)).cuda()
    g0 = torch.from_numpy(wl.random_state(shape, seed=34)[0]).cuda()
    out = {}
    for how in ("fused", "separate"):
        with fdlib.Model.from_shot(shot) as m:
            fdlib.fd_set_wavefield(m.handle, P, Po, 0)
            grad = g0.clone()
            if how == "fused":
                fdlib.fd_step_image(m.handle, lp, grad)
                torch.cuda.synchronize()
                out["after_step"] = grad.cpu().numpy()
                fdlib.fd_inject_receivers_image(m.handle, vals, lp, grad)
            else:
                fdlib.fd_step(m.handle, 1)
                fdlib.fd_imaging_product(m.handle, lp, grad)
                torch.cuda.synchronize()
                out["after_step_sep"] = grad.cpu().numpy()
                grad = g0.clone()
                fdlib.fd_step(m.handle, 0)
                # separate path of the whole update: step, inject, then one product
                fdlib.fd_set_wavefield(m.handle, P, Po, 0)
                fdlib.fd_step(m.handle, 1)
                fdlib.fd_inject_receivers(m.handle, vals)
                fdlib.fd_imaging_product(m.handle, lp, grad)
            torch.cuda.synchronize()
            out[how] = (m.wavefield(), grad.cpu().numpy())
    np.testing.assert_array_equal(out["after_step"], out["after_step_sep"])
    np.testing.assert_array_equal(out["fused"][0], out["separate"][0])
    assert pl.rel_l2(out["fused"][1], out["separate"][1]) <= 1e-6



@pytest.mark.parametrize("ndim", [2, 3])
def test_store_all_gradient_equals_checkpointed(fdlib, ndim):
    """Keeping every L'P^n (no recompute) gives the checkpointed gradient bitwise:
    the recompute reproduces the forward levels exactly."""
    import torch
    from paper_2311_05038_b300 import adjoint
    shot, vt = case(ndim, nt=90, seed=6)
    dobs = observed(fdlib, shot, vt, 3200.0)
    m = torch.from_numpy((1.0 / shot.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    out = []
    for store in (False, True):
        geo = adjoint.Geometry.from_shot(shot, checkpoint_every=25, sponge_vmax=3200.0, store_all=store)
        J, g = adjoint.misfit_and_gradient(m, geo, dobs)
        out.append((J, g.cpu().numpy()))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_store_all_entry_points_check_arguments(fdlib):
    import torch
    shape = (21, 17, 29)
    shot = _segment_case(fdlib, shape, seed=6)
    lp = torch.zeros((3,) + shape, device="cuda")
    grad = torch.zeros(shape, device="cuda")
    g = torch.zeros((3, len(shot.receivers)), device="cuda")
    with fdlib.Model.from_shot(shot) as fwd, fdlib.Model.from_shot(shot) as adj:
        fdlib.fd_step_lp_n(fwd.handle, 0, lp)                     # zero steps: nothing to do
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_step_lp_n(fwd.handle, -1, lp)
        assert e.value.status == -1
        fdlib.fd_step_lp_n(fwd.handle, 3, lp)
        assert fdlib.fd_get_step(fwd.handle) == 3
        with pytest.raises(fdlib.FDError) as e:
            fdlib.fd_adjoint_backward(adj.handle, 2, 2, lp, g, grad)
        assert e.value.status == -1
        fdlib.fd_adjoint_backward(adj.handle, 0, 3, lp, g, grad)
        assert fdlib.fd_get_step(adj.handle) == 3


def test_slowness_and_gradient_conversions_are_exact(fdlib):
    """fd_velocity_from_slowness rounds m^(-1/2) once from FP64; fd_gradient_from_image
    sums the images in array order and divides by -m in FP32: both bitwise equal to
    the same operations in NumPy."""
    import torch
    rng = np.random.default_rng(40)
    n = 100_003
    m = (1.0 / rng.uniform(1500, 4500, n) ** 2).astype(np.float32)
    v = torch.empty(n, device="cuda")
    fdlib.fd_velocity_from_slowness(torch.from_numpy(m).cuda(), v)
    np.testing.assert_array_equal(v.cpu().numpy(), (1.0 / np.sqrt(m.astype(np.float64))).astype(np.float32))
    acc = rng.standard_normal((3, n)).astype(np.float32)
    grad = torch.empty(n, device="cuda")
    fdlib.fd_gradient_from_image(torch.from_numpy(acc).cuda(), torch.from_numpy(m).cuda(), grad)
    s = (acc[0] + acc[1]) + acc[2]
    np.testing.assert_array_equal(grad.cpu().numpy(), -(s / m))
    t = torch.ones(3, device="cuda")
    assert fdlib._lib.fd_gradient_from_image(t.data_ptr(), 0, t.data_ptr(), t.data_ptr(), 3, None) == fdlib.FD_EINVAL
    assert fdlib._lib.fd_velocity_from_slowness(t.data_ptr(), None, 3, None) == fdlib.FD_EINVAL


def test_coincident_receivers_inject_deterministically(fdlib, oracle):
    """Receivers that share a point: their values are summed before the injection,
    so repeated runs agree bitwise and match the oracle's sum at that point."""
    import torch
    shape = (21, 17, 29)
    shot = _random_shot(shape, seed=41)
    shot.receivers = np.array([(5, 6, 7), (5, 6, 7), (9, 2, 3), (5, 6, 7), (9, 2, 3)], np.int32)
    vals = torch.tensor([1.0, -2.5, 0.75, 4.0, 3.0], device="cuda")
    out = []
    for _ in range(2):
        with fdlib.Model.from_shot(shot) as m:
            fdlib.fd_set_wavefield(m.handle, np.zeros(shape, np.float32), np.zeros(shape, np.float32), 0)
            lp = torch.ones(shape, device="cuda")
            grad = torch.zeros(shape, device="cuda")
            fdlib.fd_inject_receivers_image(m.handle, vals, lp, grad)
            torch.cuda.synchronize()
            out.append((m.wavefield(), grad.cpu().numpy()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    w = (shot.dt * shot.vel.astype(np.float64) / shot.h) ** 2
    emax = oracle.sponge_eta_max(float(shot.vel.max()), 3, shot.h, 1e-3)
    for (x, y, z), g in (((5, 6, 7), 1.0 - 2.5 + 4.0), ((9, 2, 3), 0.75 + 3.0)):
        a = shot.dt * (oracle.sponge_profile(shape[2], 3, emax)[x] + oracle.sponge_profile(shape[1], 3, emax)[y]
                       + oracle.sponge_profile(shape[0], 3, emax)[z])
        want = g * w[z, y, x] / (1 + a)
        assert out[0][0][z, y, x] == pytest.approx(want, rel=1e-6)
        assert out[0][1][z, y, x] == pytest.approx(want, rel=1e-6)


def _lanes_case(n=36, nt=140, nshots=3):
    shots, v_true = wl.adjoint_3d(n, nt, nshots)
    return shots, v_true, 4000.0 * 1.05


def test_shot_lanes_match_the_per_shot_gradients(fdlib):
    """ShotLanes (shots on concurrent streams, one image per lane) gives the summed
    misfit and gradient of per-shot Propagate calls, and ShotsMisfit carries it
    through autograd."""
    import torch
    from paper_2311_05038_b300 import adjoint
    shots, v_true, vmax = _lanes_case()
    geos = [adjoint.Geometry.from_shot(s, checkpoint_every=30, sponge_vmax=vmax) for s in shots]
    m = torch.from_numpy((1.0 / shots[0].vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    obs = []
    for s in shots:
        st = wl.Shot(3, s.shape, s.h, s.dt, s.nt, v_true, s.src, s.wavelet, s.receivers, sponge_width=s.sponge_width)
        with fdlib.Model.from_shot(st) as mt:
            fdlib.fd_set_sponge_vmax(mt.handle, vmax)
            mt.run_shot(s.nt)
            obs.append(torch.from_numpy(mt.traces(s.nt)).cuda())
    J_ref, g_ref = 0.0, torch.zeros_like(m)
    for geo, o in zip(geos, obs):
        J, g = adjoint.misfit_and_gradient(m, geo, o)
        J_ref += J
        g_ref += g
    lanes = adjoint.ShotLanes(geos, lanes=2)
    try:
        for _ in range(2):                       # buffers and models are reused across calls
            J, g = lanes.run(m, obs)
            assert J == pytest.approx(J_ref, rel=1e-6)
            assert pl.rel_l2(g.cpu().numpy(), g_ref.cpu().numpy()) <= 1e-6
        mm = m.clone().requires_grad_(True)
        Jt = adjoint.ShotsMisfit.apply(mm, lanes, obs)
        Jt.backward()
        assert float(Jt.detach()) == pytest.approx(J_ref, rel=1e-6)
        np.testing.assert_array_equal(mm.grad.cpu().numpy(), g.cpu().numpy())
        Jf, none = lanes.run(m, obs, backward=False)
        assert none is None and Jf == pytest.approx(J_ref, rel=1e-6)
    finally:
        lanes.close()


@pytest.mark.parametrize("data", ["zero", "anomaly"])
def test_gradient_matches_oracle_on_adjoint_workload_64(fdlib, oracle, data):
    """The adjoint workload cut down to 64^3 (its GRF model, sponge 20, +5 % anomaly
    data), 2 shots of 400 steps through ShotLanes, against the FP64 discrete
    adjoint of the oracle summed over the shots."""
    import torch
    from paper_2311_05038_b300 import adjoint
    shots, v_true = wl.adjoint_3d(64, 400, 2)
    vmax = 4000.0 * 1.05
    geos = [adjoint.Geometry.from_shot(s, checkpoint_every=50, sponge_vmax=vmax) for s in shots]
    m = torch.from_numpy((1.0 / shots[0].vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    obs = []
    for s in shots:
        if data == "zero":
            obs.append(np.zeros((s.nt, len(s.receivers))))
            continue
        _, _, tr = oracle.run(3, s.shape, s.h, s.dt, v_true, sponge_width=s.sponge_width, src=s.src,
                              wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt, sponge_vmax=vmax)
        obs.append(tr)
    lanes = adjoint.ShotLanes(geos, lanes=2)
    try:
        J, g = lanes.run(m, [torch.from_numpy(o.astype(np.float32)).cuda() for o in obs])
    finally:
        lanes.close()
    Jr, gr = 0.0, 0.0
    for s, o in zip(shots, obs):
        Js, gs, _ = oracle.misfit_gradient(3, s.shape, s.h, s.dt, velocity_of(m), sponge_width=s.sponge_width,
                                           src=s.src, wavelet=s.wavelet, receivers=s.receivers, nsteps=s.nt,
                                           observed=o.astype(np.float32).astype(np.float64), sponge_vmax=vmax)
        Jr += Js
        gr = gr + gs
    err = pl.rel_l2(g.cpu().numpy(), gr)
    print(f"64^3 adjoint workload, {data} data: misfit {J:.6e} vs {Jr:.6e}, gradient rel L2 {err:.2e}")
    assert J == pytest.approx(Jr, rel=1e-4)
    assert err <= 1e-4
