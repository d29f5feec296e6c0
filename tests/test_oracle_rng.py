"""Pins for the oracle's random-number pieces: Philox4x32-10 against its
published known-answer vectors, the project-written logarithm against libm,
and the isotropic-direction and Gaussian samplers against their
distributions."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        yield w[0:4], w[4:6], w[6:10]


def test_philox_known_answers():
    n = 0
    for ctr, key, out in _kat():
        assert O.philox4x32_10(ctr, key).tolist() == out
        n += 1
    assert n == 3


def test_philox_uniformity_chi2():
    key = [12345, 678]
    u = np.concatenate([O.philox4x32_10([i, 3, 1, 0], key) for i in range(20000)])
    hist = np.bincount((u >> 24).astype(np.int64), minlength=256)
    chi2, p = stats.chisquare(hist)
    assert p > 1e-4


@pytest.mark.parametrize("x", [1e-300, 2.2e-308, 1e-12, 0.01, 0.3, 0.70710678118654746, 0.70710678118654757,
                               0.9999999, 1.0, 1.0000001, 1.41421356, 2.0, 10.0, 1e6, 1.7e308])
def test_ln_matches_libm(x):
    ref = math.log(x)
    got = O.ln(x)
    assert abs(got - ref) <= 4 * math.ulp(ref) + 4 * math.ulp(1.0) * (abs(ref) < 1e-6)


def test_ln_random():
    rng = np.random.default_rng(1)
    xs = np.exp(rng.uniform(-40, 40, 3000))
    err = max(abs(O.ln(x) - math.log(x)) / max(math.ulp(math.log(x)), 1e-300) for x in xs)
    assert err <= 4


def test_iso_dir_distribution():
    key = [9, 9]
    d = np.array([O.iso_dir(i, 5, 2, key) for i in range(20000)])
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(d.mean(0)) < 4 / math.sqrt(3 * 20000))
    # each component of a uniform direction is uniform on [-1, 1] (Archimedes)
    for a in range(3):
        assert stats.kstest(d[:, a], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3


def test_gauss3_distribution():
    key = [4, 2]
    g = np.array([O.gauss3(i, 7, 3, key) for i in range(20000)]).reshape(-1)
    assert stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(g.var() - 1.0) < 0.03
