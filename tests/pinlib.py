"""Independent closed forms and brute-force formulations that pin the oracle.

Nothing here imports the oracle's arithmetic: coefficients come from Fornberg's
closed-form formula, the Laplacian is applied by array slicing or assembled as
a dense matrix, and the Green's functions are the textbook ones.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
from scipy import integrate


def fornberg_coefficients(r: int) -> list[Fraction]:
    """Closed form of the centred 2nd-derivative weights of radius r.

    c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!) for k >= 1, c_0 = -2 sum c_k
    (Fornberg 1988; the limit of the Lagrange-interpolation derivative).
    """
    f = math.factorial
    ck = [Fraction(2 * (-1) ** (k + 1) * f(r) ** 2, k * k * f(r - k) * f(r + k)) for k in range(1, r + 1)]
    return [-2 * sum(ck)] + ck


def read_golden_coefficients(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        out[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return out


def laplacian_sum(P: np.ndarray, c) -> np.ndarray:
    """Dimensionless stencil sum over every axis of P with a zero halo (slicing form)."""
    r = len(c) - 1
    pad = np.pad(P, r)
    core = tuple(slice(r, r + s) for s in P.shape)
    out = np.zeros_like(P, dtype=np.float64)
    for ax in range(P.ndim):
        out += float(c[0]) * P
        for k in range(1, r + 1):
            up = list(core)
            dn = list(core)
            up[ax] = slice(r + k, r + k + P.shape[ax])
            dn[ax] = slice(r - k, r - k + P.shape[ax])
            out += float(c[k]) * (pad[tuple(up)] + pad[tuple(dn)])
    return out


def toeplitz_1d(n: int, c) -> np.ndarray:
    """n x n matrix of the 1D stencil with zero halo (rows truncated at the edges)."""
    r = len(c) - 1
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = float(c[0])
        for k in range(1, r + 1):
            if i + k < n:
                A[i, i + k] = float(c[k])
            if i - k >= 0:
                A[i, i - k] = float(c[k])
    return A


def dense_laplacian(shape, c) -> np.ndarray:
    """Dense matrix of the d-axis stencil sum as a Kronecker sum of 1D matrices.

    Index order is C order over ``shape`` (last axis fastest).
    """
    mats = [toeplitz_1d(n, c) for n in shape]
    N = int(np.prod(shape))
    L = np.zeros((N, N))
    for ax in range(len(shape)):
        term = np.ones((1, 1))
        for j, n in enumerate(shape):
            term = np.kron(term, mats[ax] if j == ax else np.eye(n))
        L += term
    return L


def quad_sponge(n, W, emax):
    """Quadratic damping profile written as a vector formula (same reading as the oracle)."""
    i = np.arange(n)
    d = np.maximum(np.maximum(W - i, i - (n - 1 - W)), 0).astype(np.float64)
    return emax * (d / W) ** 2 if W > 0 else np.zeros(n)


def ricker(t, f, t0=None):
    if t0 is None:
        t0 = 1.5 / f
    a = (np.pi * f * (np.asarray(t) - t0)) ** 2
    return (1 - 2 * a) * np.exp(-a)


def green3d_ricker(r, t, c, f):
    """Field of a point source S(t) = Ricker in 3D: S(t - r/c) / (4 pi c^2 r)."""
    return ricker(t - r / c, f) / (4 * np.pi * c * c * r)


def green2d_ricker(r, t, c, f):
    """2D line-source response: (1/(2 pi c^2)) int_0^acosh(ct/r) S(t - (r/c) cosh u) du."""
    out = np.zeros(len(t))
    for i, ti in enumerate(t):
        if c * ti <= r:
            continue
        umax = math.acosh(c * ti / r)
        val, _ = integrate.quad(lambda u: float(ricker(ti - (r / c) * math.cosh(u), f)), 0.0, umax,
                                limit=200, epsabs=1e-14, epsrel=1e-12)
        out[i] = val / (2 * np.pi * c * c)
    return out


def energy(P, Pn, w, c):
    """Discrete energy E^(n+1/2) = sum (Pn-P)^2 / w - sum Pn * L'P (FP64)."""
    return float(np.sum((Pn - P) ** 2 / w) - np.sum(Pn * laplacian_sum(P, c)))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / nb) if nb > 0 else float(np.linalg.norm(a.ravel()))
