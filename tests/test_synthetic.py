"""The seeded input generators: distribution, determinism and shape (CPU only)."""
import math

import numpy as np
from scipy import stats

from synthetic import active_subset, ensemble_sizes, kepler_pair, plummer_sphere
from synthetic import rng


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 0: the published first outputs.
    z = rng.mix64(np.array([1, 2, 3], dtype=np.uint64) * rng.GAMMA)
    assert [int(c) for c in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_plummer_radii_follow_cumulative_mass_profile():
    """Plummer units: M(<r) = r^3 / (1 + r^2)^(3/2), truncated at mass fraction 0.999."""
    m, x, v = plummer_sphere(20000, 17, henon=False)
    r = np.linalg.norm(x + (m[:, None] * x).sum(0), axis=1)  # undo the tiny centre-of-mass shift
    cdf = lambda q: np.minimum(q ** 3 / (1 + q * q) ** 1.5 / 0.999, 1.0)  # noqa: E731
    assert stats.kstest(r, cdf).pvalue > 1e-3


def test_plummer_isotropy_and_centre_of_mass():
    m, x, v = plummer_sphere(20000, 18)
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-14
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-14
    u = x[:, 2] / np.linalg.norm(x, axis=1)
    assert stats.kstest(u, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert abs(m.sum() - 1) < 1e-12 and np.all(m == m[0])


def test_plummer_kinetic_energy_henon_units():
    m, x, v = plummer_sphere(20000, 19)
    ek = 0.5 * (m * (v * v).sum(1)).sum()
    assert abs(ek - 0.25) < 0.01


def test_generators_are_deterministic():
    a = plummer_sphere(1000, 5)
    b = plummer_sphere(1000, 5)
    c = plummer_sphere(1000, 6)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert not np.array_equal(a[1], c[1])


def test_active_subset():
    s = active_subset(65536, 1594, 2)
    assert s.dtype == np.int32 and len(s) == 1594 and np.all(np.diff(s) > 0)
    assert s.min() >= 0 and s.max() < 65536
    assert np.array_equal(active_subset(100, 100, 1), np.arange(100))
    assert len(active_subset(100, 0, 1)) == 0


def test_ensemble_sizes_log_uniform():
    s = ensemble_sizes(512, 4)
    assert s.min() >= 256 and s.max() < 8192
    lu = (np.log(s + 0.5) - math.log(256)) / (math.log(8192) - math.log(256))
    assert stats.kstest(lu, "uniform").pvalue > 1e-3


def test_kepler_pair_elements():
    for e in (0.0, 0.5):
        m, x, v = kepler_pair(e)
        rel = x[1] - x[0]
        assert abs(np.linalg.norm(rel) - (1 - e)) < 1e-15
        assert np.abs((m[:, None] * x).sum(0)).max() < 1e-16
        # vis-viva: v^2 = GM (2/r - 1/a)
        vr = v[1] - v[0]
        assert abs(vr @ vr - (2 / (1 - e) - 1)) < 1e-14
