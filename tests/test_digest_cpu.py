"""The CountSketch digest used to compare a full-size GPU run with the oracle's
stored run (tests/digest.py), checked against what it must satisfy."""
import numpy as np

import digest


def test_splitmix64_published_outputs():
    # SplitMix64 from state 0: the first outputs of the reference generator
    # (Steele, Lea and Flood 2014; the seeding routine of the xoshiro family).
    z = digest.splitmix64(np.arange(3, dtype=np.uint64), 0)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sketch_is_linear_and_norms_exact():
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(300_001), rng.standard_normal(300_001)
    (na, nb), (ya, yb) = digest.sketch([a, b], k=1024)
    (_,), (yd,) = digest.sketch([a - 2.5 * b], k=1024)
    np.testing.assert_allclose(ya - 2.5 * yb, yd, rtol=0, atol=1e-9)
    assert abs(na - np.linalg.norm(a)) < 1e-9 * na and abs(nb - np.linalg.norm(b)) < 1e-9 * nb


def test_sketch_estimates_relative_l2_of_typical_differences():
    """Diffuse noise, a smooth wave, a localised blob and a one-sample time shift:
    the estimate stays within 5 % of the exact relative L2 at k = 16384."""
    rng = np.random.default_rng(2)
    n = 1 << 21
    t = np.linspace(0, 60, n)
    b = np.sin(t) * np.exp(-0.02 * t) + 0.3 * np.cos(3.1 * t)
    cases = {
        "noise": b + 1e-5 * rng.standard_normal(n),
        "smooth": b * (1 + 3e-5 * np.cos(0.7 * t)),
        "blob": b + 1e-3 * np.exp(-((t - 30) / 0.05) ** 2),
        "shift": np.roll(b, 1),
    }
    (nb,), (yb,) = digest.sketch([b])
    for name, a in cases.items():
        (_,), (ya,) = digest.sketch([a])
        exact = np.linalg.norm(a - b) / np.linalg.norm(b)
        est = digest.sketch_rel_l2(ya, yb, nb)
        assert abs(est / exact - 1) < 0.05, (name, est, exact)


def test_single_changed_element_is_seen_exactly():
    b = np.linspace(-1, 1, 1_000_003)
    a = b.copy()
    a[777_777] += 3e-4
    (nb,), (yb,) = digest.sketch([b], k=4096)
    (_,), (ya,) = digest.sketch([a], k=4096)
    assert abs(digest.sketch_rel_l2(ya, yb, nb) - 3e-4 / nb) < 1e-12
