"""Compact digests of large result arrays, for comparing a full-size run with a
stored oracle run whose outputs are too large to keep (a 512^3 wavefield is 1 GB).

A digest holds the array's FP64 L2 norm and a CountSketch of it (Charikar, Chen
and Farach-Colton 2002): every element i goes to bucket ``b(i)`` with sign
``s(i)``, and ``y[j] = sum over b(i) = j of s(i) x[i]``.  The map is linear, so
for two arrays a and b, ``y(a) - y(b) = y(a - b)``, and for any array e,
``E |y(e)|^2 = |e|^2`` over the choice of hash, with relative standard deviation
at most ``sqrt(2 / k)`` for k buckets.  With k = 16384 that is about 1.1 %, so
``|y(a) - y(b)| / |b|`` estimates the relative L2 error of a against b to about
one percent of its own size.

The hash is counter-based: ``z = splitmix64(seed + (i + 1) * 0x9E3779B97F4A7C15)``
(Steele, Lea and Flood 2014, the mixing function of SplitMix64), bucket = low
bits of z (k a power of two), sign = top bit.  Nothing here is arithmetic of the
propagation method; it is a measurement used by the tests and by the script
that stores the oracle's digests.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
CHUNK = 1 << 22


def splitmix64(idx: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for counters ``idx`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def sketch(arrays, k: int = 16384, seed: int = 0x5EED):
    """(norms, sketches) of one or more arrays of the same size, in FP64.

    The arrays are flattened in C order; element i of each gets the same bucket
    and sign, so the sketches of arrays of one shape are comparable.
    """
    if k & (k - 1):
        raise ValueError("k must be a power of two")
    arrays = [np.asarray(a).reshape(-1) for a in arrays]
    n = arrays[0].size
    if any(a.size != n for a in arrays):
        raise ValueError("arrays must have the same size")
    ys = [np.zeros(k, np.float64) for _ in arrays]
    sq = [0.0 for _ in arrays]
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        z = splitmix64(np.arange(lo, hi, dtype=np.uint64), seed)
        bucket = (z & np.uint64(k - 1)).astype(np.intp)
        sign = 1.0 - 2.0 * (z >> np.uint64(63)).astype(np.float64)
        for j, a in enumerate(arrays):
            x = a[lo:hi].astype(np.float64)
            sq[j] += float(np.dot(x, x))
            ys[j] += np.bincount(bucket, weights=sign * x, minlength=k)
    return [float(np.sqrt(s)) for s in sq], ys


def sketch_rel_l2(y_a: np.ndarray, y_b: np.ndarray, norm_b: float) -> float:
    """Estimate of |a - b| / |b| from the two sketches and |b|."""
    return float(np.linalg.norm(np.asarray(y_a) - np.asarray(y_b)) / norm_b)
