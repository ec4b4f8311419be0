"""Pins of the oracle parts of the learned initialisation: the counter-based
generator, the normals, the simulation from the state-space prior and the
periodogram features.

* Philox4x32-10 against its published known-answer vectors
  (tests/golden/philox4x32_10_kat.txt).
* Normals: moments and a Kolmogorov-Smirnov test against N(0, 1).
* Simulation: the sample covariance of y over many short series equals the
  textbook Matern covariance k(t_i - t_j) + R delta_ij (a 5-sigma bound), so
  a dropped term, a wrong Cholesky factor or a wrong transition fails.
* Features: the direct transform equals numpy's FFT at frequencies that fall
  on FFT bins of an even grid; invariance to a constant shift and a scale of y.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import features as of
from oracle import model as om

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[:4], v[4:6]) == v[6:10]


def test_normals_are_standard_normal():
    z = np.concatenate([oracle.normals(11, 5, k, 4) for k in range(25_000)])
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # different series, same step: uncorrelated
    a = np.array([oracle.normals(11, 1, k, 1)[0] for k in range(20_000)])
    b = np.array([oracle.normals(11, 2, k, 1)[0] for k in range(20_000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(a.size)


@pytest.mark.parametrize("kind,nu", [("matern32", 1.5), ("matern52", 2.5)])
def test_simulated_covariance_is_the_kernel(kind, nu):
    ell, s2, R, spacing = 0.5, 1.7, 0.05, 0.3
    m = om.make_model(kind, ell, s2)
    k = om.matern_kernel(nu, ell, s2)
    N = 20_000
    Y = np.empty((N, 3))
    T = np.empty((N, 3))
    for s in range(N):
        T[s], Y[s] = oracle.simulate_series(m, R, 3, 99, s, spacing)
    assert np.all(T[:, 0] == 0.0)
    dt = np.diff(T, axis=1).ravel()
    assert abs(dt.mean() - spacing) < 5 * spacing / math.sqrt(dt.size)
    for i in range(3):
        for j in range(i, 3):
            c = Y[:, i] * Y[:, j] - (k(T[:, i] - T[:, j]) + (R if i == j else 0.0))
            assert abs(c.mean()) < 5 * c.std() / math.sqrt(N), (i, j, c.mean())


def test_features_equal_fft_on_even_grids():
    rng = np.random.default_rng(1)
    n = 4096
    w = of.frequencies()
    y = rng.normal(size=n) + np.cos(w[10] * 0.01 * np.arange(n))
    for j, mbin in ((10, 50), (40, 700)):
        dt = 2 * math.pi * mbin / (n * w[j])         # w_j falls on FFT bin mbin
        t = dt * np.arange(n)
        f = of.features(t, y)
        yc = y - y.mean()
        P = abs(np.fft.fft(yc)[mbin]) ** 2 / (n * np.mean(yc * yc))
        assert abs(f[j] - math.log(P + 1e-8)) < 1e-9
    assert abs(f[64] - math.log(np.var(y))) < 1e-12


def test_features_invariances_and_edge_cases():
    rng = np.random.default_rng(2)
    t = np.cumsum(rng.exponential(0.01, 3000))
    y = rng.normal(size=3000)
    f = of.features(t, y)
    g = of.features(t, 3.0 * y + 5.0)
    assert np.allclose(f[:64], g[:64], atol=1e-10)
    assert abs(g[64] - f[64] - math.log(9.0)) < 1e-12
    assert np.all(of.features(t, np.ones(3000)) == 0.0)
    # white noise: the normalised periodogram averages to 1 over the bins
    assert abs(np.mean(np.exp(f[:64])) - 1.0) < 0.35
