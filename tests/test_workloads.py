"""The seeded input generators against the distributions they claim (Sec. III:
"Cube", "Sphere" and "Plummer" particle sets).  Each check is a closed form or
a Kolmogorov-Smirnov test at fixed seeds, so the outcome is deterministic."""

import numpy as np
import pytest
from scipy import stats

from paper_1405_7487_gb300 import workloads as W

N = 200_000


def _ks(sample, cdf):
    return stats.kstest(np.asarray(sample, np.float64), cdf).pvalue


def test_seeded_and_float32():
    for f in (W.cube, W.plummer, W.sphere):
        a, b, c = f(1000, 5), f(1000, 5), f(1000, 6)
        assert a.dtype == np.float32 and a.shape == (1000, 4)
        assert np.array_equal(a, b) and not np.array_equal(a, c)
    w = W.weights(1000, 40)
    assert w.dtype == np.float32 and np.array_equal(w, W.weights(1000, 40))


def test_cube_uniform():
    x = W.cube(N, 11).astype(np.float64)
    assert np.all((x[:, :3] >= 0) & (x[:, :3] <= 1)) and np.all((x[:, 3] >= -1) & (x[:, 3] <= 1))
    for a in range(3):
        assert _ks(x[:, a], stats.uniform(0, 1).cdf) > 1e-3
    assert _ks(x[:, 3], stats.uniform(-1, 2).cdf) > 1e-3


def _isotropic(u):
    # uniform directions: cos(polar angle) and the azimuth are uniform
    ct = u[:, 2] / np.linalg.norm(u, axis=1)
    az = np.arctan2(u[:, 1], u[:, 0])
    assert _ks(ct, stats.uniform(-1, 2).cdf) > 1e-3
    assert _ks(az, stats.uniform(-np.pi, 2 * np.pi).cdf) > 1e-3


def test_sphere_surface():
    x = W.sphere(N, 12).astype(np.float64)
    r = np.linalg.norm(x[:, :3], axis=1)
    assert np.all(np.abs(r - 1.0) < 1e-6)
    _isotropic(x[:, :3])
    assert _ks(x[:, 3], stats.uniform(-1, 2).cdf) > 1e-3


def test_plummer_mass_profile():
    # Plummer's enclosed mass M(<r) = r^3 / (r^2 + a^2)^(3/2), truncated at
    # r_max = 20 and renormalised
    a, rmax = 1.0, 20.0
    x = W.plummer(N, 13).astype(np.float64)
    r = np.linalg.norm(x[:, :3], axis=1)
    assert r.max() <= rmax * (1 + 1e-6)
    M = lambda s: s ** 3 / (s * s + a * a) ** 1.5  # noqa: E731
    cdf = lambda s: M(np.clip(s, 0, rmax)) / M(rmax)  # noqa: E731
    assert _ks(r, cdf) > 1e-3
    # half of the (untruncated) mass lies within r = a / sqrt(2^(2/3) - 1) ~ 1.305 a
    r_half = a / np.sqrt(2 ** (2 / 3) - 1)
    assert np.mean(r < r_half) == pytest.approx(0.5 / M(rmax), abs=0.005)
    _isotropic(x[:, :3])
    assert np.all(x[:, 3] == np.float32(1.0 / N))


def test_sample_targets():
    t = W.sample_targets(10_000, 4096)
    assert t.dtype == np.int64 and t.shape == (4096,)
    assert np.unique(t).size == 4096 and t.min() >= 0 and t.max() < 10_000
    assert np.array_equal(t, W.sample_targets(10_000, 4096))
    assert W.sample_targets(100, 4096).shape == (100,)
