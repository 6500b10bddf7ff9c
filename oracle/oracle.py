"""FP64 CPU oracle for the acoustic finite-difference propagator.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
module.  It shares no code with the CUDA library: it derives its own stencil
coefficients (exact rational Taylor solve), its own sponge profiles and its own
stability limit, and runs a plain FP64 loop (``fd_oracle.c``).

What it computes follows the paper's proof-of-concept (section 7): Eq. 1,
``P_tt = v^2 (P_xx + P_zz) + S(t)``, advanced by the routine sequence of the
WaveSimulator listing (add_source, fd_pzz, fd_pxx, fd_time, swap, swap).  The
paper does not fix the stencil order, the boundary, the sponge, the source
scaling or the receivers; the readings taken here are:

* stencil: radius 4 (8th order), coefficients from the Taylor conditions;
* boundary: P = 0 outside the grid (zero halo, "rigid");
* sponge: damped leapfrog ``Pn = (2P - (1-a) Pold + w L'P) / (1+a)`` with
  ``a = dt (eta_x + eta_y + eta_z)``, each 1D profile ``eta_max (d/W)^2`` over a
  W-point band, ``eta_max = 3 v_max ln(1/R) / (2 W h)``;
* source: ``Pn[src] += dt^2 S(t_n) / h^d`` after the update of step n;
* receivers: ``trace[n] = Pn[rec]``, the field at ``t_{n+1}``.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed
forms (Fornberg's coefficient formula, convergence orders, Green's functions,
discrete energy, reciprocity, the CFL limit, a dense-matrix brute force).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RADIUS = 4


# --------------------------------------------------------------------------- build

def build(force: bool = False) -> str:
    """Compile fd_oracle.c into liboracle.so with gcc (OpenMP on the z loop)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _configure(lib):
    """Declare the C signatures on a loaded liboracle."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.fdo_run.restype = ctypes.c_int
    lib.fdo_run.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,       # ndim nx ny nz
        ctypes.c_double, ctypes.c_double,                            # h dt
        ctypes.c_int, dp, dp,                                        # radius c vel
        dp, dp, dp,                                                  # eta_x eta_y eta_z
        ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,  # src, wavelet, nt_w
        ctypes.c_int, ip,                                            # nrec rec_xyz
        dp, dp, ctypes.c_int, ctypes.c_int,                          # P Pold n0 nsteps
        dp, ctypes.c_int]                                            # traces nthreads
    lib.fdo_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def max_threads() -> int:
    """Threads the oracle's OpenMP loop uses by default on this host."""
    return int(_load().fdo_max_threads())


# --------------------------------------------------------------- stencil coefficients

def taylor_coefficients(radius: int = RADIUS) -> list[Fraction]:
    """Exact coefficients c_0..c_r of the centred stencil for h^2 d^2/dx^2.

    Expanding ``c_0 f(0) + sum_k c_k (f(kh) + f(-kh))`` in Taylor series gives
    ``(c_0 + 2 sum c_k) f + 2 sum_j (sum_k c_k k^(2j)) h^(2j) f^(2j) / (2j)!``.
    Matching ``h^2 f''`` to the highest order reachable with r unknowns asks
    ``sum_k c_k k^2 = 1`` and ``sum_k c_k k^(2j) = 0`` for j = 2..r, then
    ``c_0 = -2 sum_k c_k``.  The r x r system is solved by Gaussian elimination
    in exact rational arithmetic.
    """
    r = int(radius)
    if r < 1:
        raise ValueError("radius must be >= 1")
    # rows j = 1..r, columns k = 1..r: A[j][k] = k^(2j); rhs = [1, 0, ..., 0]
    A = [[Fraction(k) ** (2 * j) for k in range(1, r + 1)] for j in range(1, r + 1)]
    b = [Fraction(1)] + [Fraction(0)] * (r - 1)
    for col in range(r):
        piv = next(i for i in range(col, r) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for i in range(r):
            if i != col and A[i][col] != 0:
                f = A[i][col] / A[col][col]
                A[i] = [a - f * p for a, p in zip(A[i], A[col])]
                b[i] -= f * b[col]
    ck = [b[i] / A[i][i] for i in range(r)]
    c0 = -2 * sum(ck)
    return [c0] + ck


def coefficients_f64(radius: int = RADIUS) -> np.ndarray:
    """The Taylor coefficients as FP64 values."""
    return np.array([float(x) for x in taylor_coefficients(radius)], dtype=np.float64)


def cfl_limit(ndim: int, radius: int = RADIUS) -> float:
    """Largest stable Courant number v_max dt / h of the leapfrog scheme.

    The stencil's symbol is ``c_0 + 2 sum_k c_k cos(k theta)``; its most negative
    value is at theta = pi, ``-lambda_1`` with
    ``lambda_1 = -(c_0 + 2 sum_k (-1)^k c_k)``.  The leapfrog for
    ``u'' = -omega^2 u`` is stable for ``omega dt <= 2``, and on d axes
    ``omega^2 <= d lambda_1 v^2 / h^2``, so ``C <= 2 / sqrt(d lambda_1)``.
    """
    c = taylor_coefficients(radius)
    lam1 = -(c[0] + 2 * sum(((-1) ** k) * c[k] for k in range(1, len(c))))
    return 2.0 / math.sqrt(ndim * float(lam1))


# ------------------------------------------------------------------------- sponge

def sponge_eta_max(v_max: float, width: int, h: float, R: float) -> float:
    """Peak damping rate (1/s) of a width-W quadratic sponge with target reflection R."""
    if width <= 0:
        return 0.0
    return 3.0 * v_max * math.log(1.0 / R) / (2.0 * width * h)


def sponge_profile(n: int, width: int, eta_max: float) -> np.ndarray:
    """1D damping-rate profile (1/s) along an axis of n points.

    Point i lies ``d = max(W - i, i - (n - 1 - W), 0)`` points into the band,
    so the outermost point has d = W, the innermost band point d = 1 and the
    interior d = 0; the rate is ``eta_max (d / W)^2``.
    """
    eta = np.zeros(n, dtype=np.float64)
    if width <= 0:
        return eta
    for i in range(n):
        d = max(width - i, i - (n - 1 - width), 0)
        eta[i] = eta_max * (d / width) ** 2
    return eta


# ----------------------------------------------------------------------- propagate

def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def run(ndim: int, shape, h: float, dt: float, vel, *, sponge_width: int = 0,
        sponge_R: float = 1e-3, src=None, wavelet=None, receivers=None,
        P=None, Pold=None, n0: int = 0, nsteps: int = 0, nthreads: int = 0,
        coefficients=None, sponge_vmax=None):
    """Advance the FP64 scheme by ``nsteps`` steps; returns (P, Pold, traces).

    shape      (nz, nx) in 2D, (nz, ny, nx) in 3D; arrays are x-fastest.
    vel        velocities (m/s), any float dtype, converted exactly to FP64.
    src        source point (ix, iy, iz), with ``wavelet`` = S(t_n); iy is
               ignored in 2D.
    receivers  int array [nrec, 3] of (ix, iy, iz); iy ignored in 2D.
    P, Pold    initial levels n0 and n0-1 (default zero).
    coefficients  override c_0..c_r (default: the Taylor coefficients); only the
               pin tests pass this.
    sponge_vmax  velocity that sets the sponge strength (default: the largest
               velocity of the model).
    """
    lib = _load()
    if ndim == 2:
        nz, nx = shape
        ny = 1
    elif ndim == 3:
        nz, ny, nx = shape
    else:
        raise ValueError("ndim must be 2 or 3")
    npts = nz * ny * nx
    v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64).reshape(npts))
    c = np.ascontiguousarray(coefficients if coefficients is not None else coefficients_f64(),
                             dtype=np.float64)
    radius = len(c) - 1
    Pa = np.zeros(npts) if P is None else np.array(P, dtype=np.float64).reshape(npts).copy()
    Po = np.zeros(npts) if Pold is None else np.array(Pold, dtype=np.float64).reshape(npts).copy()
    etas = [None, None, None]
    if sponge_width > 0:
        vm = float(v.max()) if sponge_vmax is None else float(sponge_vmax)
        em = sponge_eta_max(vm, sponge_width, h, sponge_R)
        etas = [sponge_profile(nx, sponge_width, em),
                sponge_profile(ny, sponge_width, em) if ndim == 3 else None,
                sponge_profile(nz, sponge_width, em)]
    six = siy = siz = 0
    wav = None
    ntw = 0
    if src is not None and wavelet is not None:
        six, siy, siz = (int(q) for q in src)
        if ndim == 2:
            siy = 0
        wav = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float64))
        ntw = len(wav)
    nrec = 0
    rec = None
    if receivers is not None and len(receivers):
        rec = np.ascontiguousarray(np.asarray(receivers, dtype=np.int32).reshape(-1, 3))
        if ndim == 2:
            rec = rec.copy()
            rec[:, 1] = 0
        nrec = len(rec)
    traces = np.zeros((nsteps, nrec), dtype=np.float64) if nrec else None
    st = lib.fdo_run(ndim, nx, ny, nz, float(h), float(dt), radius, _dp(c), _dp(v),
                     _dp(etas[0]), _dp(etas[1]), _dp(etas[2]),
                     six, siy, siz, _dp(wav), ntw,
                     nrec, None if rec is None else rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     _dp(Pa), _dp(Po), int(n0), int(nsteps), _dp(traces), int(nthreads))
    if st != 0:
        raise ValueError(f"fdo_run rejected its arguments (status {st})")
    return Pa.reshape(shape), Po.reshape(shape), traces


# ------------------------------------------------------------------------ adjoint

def stencil_sum(P: np.ndarray, coefficients=None) -> np.ndarray:
    """L'P: sum over the axes of c_0 P + sum_k c_k (P[+k] + P[-k]), zero outside (FP64)."""
    c = coefficients_f64() if coefficients is None else np.asarray(coefficients, np.float64)
    r = len(c) - 1
    pad = np.pad(np.asarray(P, np.float64), r)
    core = tuple(slice(r, r + n) for n in P.shape)
    out = np.zeros(P.shape, np.float64)
    for ax in range(P.ndim):
        out += c[0] * P
        for k in range(1, r + 1):
            up = list(core)
            dn = list(core)
            up[ax] = slice(r + k, r + k + P.shape[ax])
            dn[ax] = slice(r - k, r - k + P.shape[ax])
            out += c[k] * (pad[tuple(up)] + pad[tuple(dn)])
    return out


def misfit_gradient(ndim: int, shape, h: float, dt: float, vel, *, sponge_width: int = 0,
                    sponge_R: float = 1e-3, src=None, wavelet=None, receivers=None, nsteps: int = 0,
                    observed=None, sponge_vmax=None):
    """J = 1/2 sum_n |d^n - observed^n|^2 and dJ/dm (m = 1/v^2), FP64, by the discrete adjoint.

    The forward recurrence (1+a) P^{n+1} = 2P^n - (1-a) P^{n-1} + W L'P^n + (1+a) s^n e_src,
    d^n = R P^{n+1}, W = diag((dt v / h)^2) has, for g^n = d^n - observed^n, the adjoint
    (with psi = W lambda / (1+a))
        (1+a) psi_k = 2 psi_{k+1} - (1-a) psi_{k+2} + W L'psi_{k+1} + W R^T g^{k-1},
    k = nt .. 1, psi_{nt+1} = psi_{nt+2} = 0, and the gradient
        dJ/dm = -(1/m) sum_{n=0}^{nt-1} psi_{n+1} L'P^n.
    The damping a is held fixed (its strength comes from sponge_vmax).  Every
    forward level is kept, so this is for small grids.  Returns (J, grad_m, traces).
    """
    v = np.asarray(vel, np.float64).reshape(shape)
    vmax = float(v.max()) if sponge_vmax is None else float(sponge_vmax)
    rec = np.asarray(receivers, np.int64).reshape(-1, 3)
    P = np.zeros(shape)
    Pold = np.zeros(shape)
    levels = [P.copy()]                        # P^0 .. P^{nt-1}
    traces = np.zeros((nsteps, len(rec)))
    for n in range(nsteps):
        P, Pold, tr = run(ndim, shape, h, dt, v, sponge_width=sponge_width, sponge_R=sponge_R, src=src,
                          wavelet=wavelet, receivers=rec, P=P, Pold=Pold, n0=n, nsteps=1, sponge_vmax=vmax)
        traces[n] = tr[0]
        if n + 1 < nsteps:
            levels.append(P.copy())
    g = traces - np.asarray(observed, np.float64)
    J = 0.5 * float(np.sum(g * g))
    # receiver points and their w / (1 + a)
    w = (dt * v / h) ** 2
    a = np.zeros(shape)
    if sponge_width > 0:
        em = sponge_eta_max(vmax, sponge_width, h, sponge_R)
        a = a + dt * sponge_profile(shape[-1], sponge_width, em)
        a = a + dt * sponge_profile(shape[0], sponge_width, em).reshape((shape[0],) + (1,) * (ndim - 1))
        if ndim == 3:
            a = a + dt * sponge_profile(shape[1], sponge_width, em).reshape((1, shape[1], 1))
    if ndim == 2:
        pts = (rec[:, 2], rec[:, 0])
    else:
        pts = (rec[:, 2], rec[:, 1], rec[:, 0])
    scale = w[pts] / (1.0 + a[pts])
    psi = np.zeros(shape)         # psi_{k+1}
    psi_old = np.zeros(shape)     # psi_{k+2}
    acc = np.zeros(shape)
    for k in range(nsteps, 0, -1):
        nxt, _, _ = run(ndim, shape, h, dt, v, sponge_width=sponge_width, sponge_R=sponge_R,
                        P=psi, Pold=psi_old, nsteps=1, sponge_vmax=vmax)
        np.add.at(nxt, pts, scale * g[k - 1])
        psi_old, psi = psi, nxt
        acc += psi * stencil_sum(levels[k - 1])
    m = 1.0 / (v * v)
    return J, -acc / m, traces
