"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: Fornberg's
closed form and published table for the stencil weights, the convergence order
of the operator and of the scheme, the homogeneous-medium Green's functions
(3D closed form, 2D quadrature), the exact discrete energy identity with and
without the sponge, source-receiver reciprocity, the leapfrog stability limit,
and a dense-matrix brute force of the whole recurrence on tiny grids.
"""
import math
import os

import numpy as np
import pytest

import pinlib as pl
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- coefficients

@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_taylor_coefficients_equal_fornberg_closed_form(oracle, r):
    assert oracle.taylor_coefficients(r) == pl.fornberg_coefficients(r)


def test_taylor_coefficients_equal_published_table(oracle):
    table = pl.read_golden_coefficients(os.path.join(GOLDEN, "fd_coefficients.txt"))
    assert set(table) == {1, 2, 3, 4}
    for r, coeffs in table.items():
        assert oracle.taylor_coefficients(r) == coeffs


def test_radius4_table():
    # the 8th-order weights used on every axis
    from fractions import Fraction as F
    assert pl.fornberg_coefficients(4) == [F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)]


# ----------------------------------------------------------------- operator order

def _one_step_laplacian(oracle, f, h):
    """Recover L'f from one oracle step: P = Pold = f, w = 1 gives Pn = f + L'f."""
    dt = 1e-3
    v = np.full(f.shape, h / dt)          # (dt v / h)^2 = 1
    P, _, _ = oracle.run(f.ndim, f.shape, h, dt, v, P=f, Pold=f, nsteps=1)
    return P - f


def test_operator_is_eighth_order(oracle):
    """Error of (1/h^2) L' on a Gaussian falls as h^8 under refinement."""
    sigma = 1.0
    errs = []
    for m in (4, 8):                       # points per sigma
        h = sigma / m
        x = np.arange(-10 * m, 10 * m + 1) * h
        X, Z = np.meshgrid(x, x, indexing="xy")
        g = np.exp(-(X ** 2 + Z ** 2) / (2 * sigma ** 2))
        exact = g * ((X ** 2 + Z ** 2) / sigma ** 4 - 2 / sigma ** 2)
        lap = _one_step_laplacian(oracle, g, h) / h ** 2
        errs.append(np.max(np.abs(lap - exact)) / np.max(np.abs(exact)))
    order = math.log2(errs[0] / errs[1])
    assert 7.6 < order < 8.6, (errs, order)


def test_operator_is_axis_symmetric_3d(oracle):
    """Applying L' to f(x), f(y), f(z) gives the same values (every axis present)."""
    rng = np.random.default_rng(0)
    prof = rng.standard_normal(12)
    n = 12
    fx = np.broadcast_to(prof[None, None, :], (n, n, n)).copy()
    fy = np.broadcast_to(prof[None, :, None], (n, n, n)).copy()
    fz = np.broadcast_to(prof[:, None, None], (n, n, n)).copy()
    lx = _one_step_laplacian(oracle, fx, 1.0)
    ly = _one_step_laplacian(oracle, fy, 1.0)
    lz = _one_step_laplacian(oracle, fz, 1.0)
    np.testing.assert_allclose(lx, np.transpose(ly, (0, 2, 1)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(lx, np.transpose(lz, (2, 1, 0)), rtol=0, atol=1e-12)


# ----------------------------------------------------------------- scheme order

def test_scheme_is_second_order_in_time(oracle):
    """Fixed Courant number, h and dt halved together: differences shrink 4x.

    The initial levels are the exact solution at t = 0 and t = -dt to O(dt^4)
    (Taylor series with the analytic Laplacians of the Gaussian), so the global
    error is the scheme's own O(dt^2 + h^8).
    """
    c, sigma, L, T = 2000.0, 60.0, 1280.0, 0.2
    sols = []
    for h in (20.0, 10.0, 5.0):
        x = np.arange(-L, L + h / 2, h)
        X, Z = np.meshgrid(x, x, indexing="xy")
        rho2 = (X ** 2 + Z ** 2) / sigma ** 2
        g = np.exp(-rho2 / 2)
        lap_g = g * (rho2 - 2) / sigma ** 2
        lap2_g = g * (rho2 ** 2 - 8 * rho2 + 8) / sigma ** 4
        dt = 0.4 * h / c
        Pm1 = g + (dt * c) ** 2 / 2 * lap_g + (dt * c) ** 4 / 24 * lap2_g
        nsteps = int(round(T / dt))
        P, _, _ = oracle.run(2, g.shape, h, dt, np.full(g.shape, c), P=g, Pold=Pm1, nsteps=nsteps)
        sols.append(P)
    coarse = sols[0]
    mid = sols[1][::2, ::2]
    fine = sols[2][::4, ::4]
    d1 = np.linalg.norm(coarse - mid)
    d2 = np.linalg.norm(mid - fine)
    order = math.log2(d1 / d2)
    assert 1.8 < order < 2.2, (d1, d2, order)


# ----------------------------------------------------------------- energy

def _hetero_velocity(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1500.0, 4000.0, shape).astype(np.float32)


@pytest.mark.parametrize("shape", [(40, 56), (14, 12, 18)])
def test_energy_is_conserved_without_sponge(oracle, shape):
    """Zero halo, no sponge, no source: E^(n+1/2) is constant to rounding."""
    ndim = len(shape)
    h = 10.0
    v = _hetero_velocity(shape, 7)
    dt = 0.4 * h / float(v.max())
    rng = np.random.default_rng(8)
    P = rng.standard_normal(shape)
    Pold = rng.standard_normal(shape)
    c = pl.fornberg_coefficients(4)
    w = (dt * v.astype(np.float64) / h) ** 2
    E = []
    for _ in range(50):
        Pn, Pc, _ = oracle.run(ndim, shape, h, dt, v, P=P, Pold=Pold, nsteps=20)
        # Pn is level m+1, Pc level m
        E.append(pl.energy(Pc, Pn, w, c))
        P, Pold = Pn, Pc
    E = np.array(E)
    assert np.all(E > 0)
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-11, E


def test_energy_identity_with_sponge(oracle):
    """With damping a: E^(n+1/2) - E^(n-1/2) = -sum (a / w) (Pn - Pold)^2 exactly."""
    shape = (36, 44)
    h = 10.0
    W = 8
    v = _hetero_velocity(shape, 9)
    dt = 0.4 * h / float(v.max())
    rng = np.random.default_rng(10)
    P0 = rng.standard_normal(shape)
    Pm1 = rng.standard_normal(shape)
    c = pl.fornberg_coefficients(4)
    w = (dt * v.astype(np.float64) / h) ** 2
    emax = 3.0 * float(v.max()) * math.log(1e3) / (2.0 * W * h)
    a = dt * (pl.quad_sponge(shape[1], W, emax)[None, :] + pl.quad_sponge(shape[0], W, emax)[:, None])
    levels = [Pm1, P0]
    P, Pold = P0, Pm1
    for _ in range(30):
        P, Pold, _ = oracle.run(2, shape, h, dt, v, sponge_width=W, sponge_R=1e-3,
                                P=P, Pold=Pold, nsteps=1)
        levels.append(P)
    Es = [pl.energy(levels[i], levels[i + 1], w, c) for i in range(len(levels) - 1)]
    for n in range(1, len(Es)):
        loss = np.sum(a / w * (levels[n + 1] - levels[n - 1]) ** 2)
        assert loss > 0
        assert abs((Es[n] - Es[n - 1]) + loss) <= 1e-11 * Es[0], (n, Es[n] - Es[n - 1], loss)


def test_sponge_profile_integral_matches_reflection_target(oracle):
    """exp(-(2/c) int eta dx) over the band equals R for the quadratic profile."""
    W, h, v, R = 20, 10.0, 3000.0, 1e-3
    emax = oracle.sponge_eta_max(v, W, h, R)
    prof = oracle.sponge_profile(200, W, emax)
    assert prof[0] == pytest.approx(emax) and prof[-1] == pytest.approx(emax)
    assert prof[W - 1] == pytest.approx(emax / W ** 2)
    assert np.all(prof[W:200 - W] == 0)
    np.testing.assert_allclose(prof, prof[::-1])
    # the band samples eta_max (s/L)^2 at s = d h, d = W..0 (i = 0..W); its
    # trapezoid integral is eta_max L / 3 + O(h^2), and exp(-(2/c) int eta) = R
    integral = h * (np.sum(prof[:W + 1]) - 0.5 * (prof[0] + prof[W]))
    assert integral == pytest.approx(emax * W * h / 3.0, rel=5e-3)
    refl = math.exp(-2.0 * integral / v)
    assert refl == pytest.approx(R, rel=2e-2)


def test_sponge_absorbs_outgoing_wave(oracle):
    """A pulse leaving through the sponge loses > 99% of its energy; without it, none."""
    n, h, W = 120, 10.0, 20
    v = np.full((n, n), 2000.0, dtype=np.float32)
    dt = 0.4 * h / 2000.0
    x = (np.arange(n) - n / 2) * h
    X, Z = np.meshgrid(x, x, indexing="xy")
    g = np.exp(-(X ** 2 + Z ** 2) / (2 * 30.0 ** 2))
    c = pl.fornberg_coefficients(4)
    w = (dt * v.astype(np.float64) / h) ** 2
    steps = int(1.2 / dt)
    out = {}
    for width in (0, W):
        P, Pold, _ = oracle.run(2, (n, n), h, dt, v, sponge_width=width, P=g, Pold=g, nsteps=1)
        E0 = pl.energy(Pold, P, w, c)
        P2, Pold2, _ = oracle.run(2, (n, n), h, dt, v, sponge_width=width, P=P, Pold=Pold, nsteps=steps)
        out[width] = pl.energy(Pold2, P2, w, c) / E0
    assert out[0] == pytest.approx(1.0, abs=1e-9)
    assert out[W] < 1e-2, out


# ----------------------------------------------------------------- Green's functions

def test_green_function_3d(oracle):
    """Homogeneous 3D point source: trace = S(t - r/c) / (4 pi c^2 r) before reflections."""
    n, h, c, f = 112, 10.0, 2000.0, 10.0
    dt = 0.4 * h / c
    nt = 240
    s = n // 2
    rec = np.array([(s + k, s, s) for k in (15, 20, 25)], dtype=np.int32)
    wav = wl.ricker(nt, dt, f)
    _, _, tr = oracle.run(3, (n, n, n), h, dt, np.full((n, n, n), c, np.float32), src=(s, s, s),
                          wavelet=wav, receivers=rec, nsteps=nt)
    t = (np.arange(nt) + 1) * dt                       # trace[n] is the field at t_(n+1)
    for j, k in enumerate((15, 20, 25)):
        r = k * h
        ana = pl.green3d_ricker(r, t, c, f)
        # compare in the window before the first boundary reflection (path 2 s h - r)
        win = t < (2 * s * h - r) / c - 0.02
        err = pl.rel_l2(tr[win, j], ana[win])
        assert err < 0.03, (k, err)
        # a one-sample timing error would cost ~15% here
        late = pl.rel_l2(tr[win, j], pl.green3d_ricker(r, t[win] - dt, c, f))
        assert late > 4 * err, (k, err, late)


def test_green_function_2d_and_refinement(oracle):
    """Homogeneous 2D line source: trace matches the quadrature; error drops ~4x per halving."""
    c, f = 2000.0, 15.0
    errs = []
    for h, n in ((10.0, 256), (5.0, 512)):
        dt = 0.4 * h / c
        T = 0.6
        nt = int(round(T / dt))
        s = n // 2
        k = int(round(480.0 / h))
        rec = np.array([(s + k, 0, s)], dtype=np.int32)
        wav = wl.ricker(nt, dt, f)
        _, _, tr = oracle.run(2, (n, n), h, dt, np.full((n, n), c, np.float32), src=(s, 0, s),
                              wavelet=wav, receivers=rec, nsteps=nt)
        t = (np.arange(nt) + 1) * dt
        ana = pl.green2d_ricker(480.0, t, c, f)
        errs.append(pl.rel_l2(tr[:, 0], ana))
    assert errs[0] < 0.08, errs
    assert errs[0] / errs[1] > 3.0, errs


# ----------------------------------------------------------------- reciprocity

@pytest.mark.parametrize("ndim,width", [(2, 0), (2, 6), (3, 4)])
def test_reciprocity(oracle, ndim, width):
    """v(x_s)^2 P_(s->r)(t) = v(x_r)^2 P_(r->s)(t) on a heterogeneous model."""
    shape = (34, 40) if ndim == 2 else (18, 20, 22)
    h = 10.0
    v = _hetero_velocity(shape, 11)
    dt = 0.4 * h / float(v.max())
    nt = 150
    wav = wl.ricker(nt, dt, 25.0)
    if ndim == 2:
        a, b = (12, 0, 11), (27, 0, 22)
        va, vb = v[a[2], a[0]], v[b[2], b[0]]
    else:
        a, b = (6, 7, 6), (15, 12, 11)
        va, vb = v[a[2], a[1], a[0]], v[b[2], b[1], b[0]]
    _, _, ab = oracle.run(ndim, shape, h, dt, v, sponge_width=width, src=a, wavelet=wav,
                          receivers=np.array([b], np.int32), nsteps=nt)
    _, _, ba = oracle.run(ndim, shape, h, dt, v, sponge_width=width, src=b, wavelet=wav,
                          receivers=np.array([a], np.int32), nsteps=nt)
    lhs = float(va) ** 2 * ab[:, 0]
    rhs = float(vb) ** 2 * ba[:, 0]
    assert np.max(np.abs(lhs)) > 0
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))
    # and the relation is not trivially symmetric: the raw traces differ when v differs
    assert abs(float(va) - float(vb)) > 1.0
    assert np.max(np.abs(ab - ba)) > 1e-3 * np.max(np.abs(ab))


# ----------------------------------------------------------------- CFL

def test_cfl_limit_value(oracle):
    assert oracle.cfl_limit(2) == pytest.approx(0.55463, abs=1e-4)
    assert oracle.cfl_limit(3) == pytest.approx(0.45286, abs=1e-4)


@pytest.mark.parametrize("ndim,shape,steps", [(2, (64, 64), 10000), (3, (24, 24, 24), 3000)])
def test_cfl_limit_separates_stable_from_unstable(oracle, ndim, shape, steps):
    h, v0 = 10.0, 2000.0
    rng = np.random.default_rng(3)
    P0 = rng.standard_normal(shape)
    lim = oracle.cfl_limit(ndim)
    grow = {}
    for frac in (0.99, 1.01):
        dt = frac * lim * h / v0
        P, _, _ = oracle.run(ndim, shape, h, dt, np.full(shape, v0), P=P0, Pold=P0, nsteps=steps)
        grow[frac] = np.max(np.abs(P)) / np.max(np.abs(P0))
    assert grow[0.99] < 10.0, grow
    assert not np.isfinite(grow[1.01]) or grow[1.01] > 1e6, grow


# ----------------------------------------------------------------- brute force

@pytest.mark.parametrize("shape,width", [((9, 11), 0), ((9, 11), 3), ((7, 9, 11), 2)])
def test_dense_matrix_brute_force(oracle, shape, width):
    """The whole recurrence written with a dense Laplacian matrix agrees to 1e-13."""
    ndim = len(shape)
    h = 10.0
    v = _hetero_velocity(shape, 12).astype(np.float64)
    dt = 0.35 * h / float(v.max())
    nt = 20
    rng = np.random.default_rng(13)
    wav = rng.standard_normal(nt).astype(np.float32)
    src = (4, 0, 5) if ndim == 2 else (4, 3, 2)
    recs = np.array([(1, 0, 2), (8, 0, 7), (src[0], src[1], src[2])], np.int32) if ndim == 2 else \
        np.array([(1, 2, 3), (8, 6, 5), (src[0], src[1], src[2])], np.int32)
    P0 = rng.standard_normal(shape)
    Pm1 = rng.standard_normal(shape)
    Po, _, tro = oracle.run(ndim, shape, h, dt, v.astype(np.float32), sponge_width=width,
                            src=src, wavelet=wav, receivers=recs, P=P0, Pold=Pm1, nsteps=nt)
    # dense formulation
    c = pl.fornberg_coefficients(4)
    Lm = pl.dense_laplacian(shape, c)
    vv = v.astype(np.float32).astype(np.float64).ravel()
    w = (dt * vv / h) ** 2
    emax = 3.0 * vv.max() * math.log(1e3) / (2.0 * width * h) if width else 0.0
    prof = [pl.quad_sponge(nn, width, emax) for nn in shape]
    eta = np.zeros(shape)
    for ax, p in enumerate(prof):
        sh = [1] * ndim
        sh[ax] = len(p)
        eta = eta + p.reshape(sh)
    a = dt * eta.ravel()
    def flat(pt):
        ix, iy, iz = pt
        return (iz * shape[1] + ix) if ndim == 2 else ((iz * shape[1] + iy) * shape[2] + ix)
    P = P0.ravel().copy()
    Pold = Pm1.ravel().copy()
    tr = np.zeros((nt, len(recs)))
    for n in range(nt):
        Pn = (2 * P - (1 - a) * Pold + w * (Lm @ P)) / (1 + a)
        Pn[flat(src)] += dt * dt * float(wav[n]) / h ** ndim
        tr[n] = [Pn[flat(r)] for r in recs]
        Pold, P = P, Pn
    scale = np.max(np.abs(P))
    assert np.max(np.abs(Po.ravel() - P)) <= 1e-13 * scale
    assert np.max(np.abs(tro - tr)) <= 1e-13 * np.max(np.abs(tr))
