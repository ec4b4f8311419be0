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


def test_dft_power_equals_fft_bins():
    """On the regular grid, A(w) at w = 2 pi m / (n dbar) is FFT bin m."""
    rng = np.random.default_rng(1)
    n = 4096
    y = rng.normal(size=n) + np.cos(0.3 * np.arange(n))
    dbar = 0.01
    yc = y - y.mean()
    F = np.fft.fft(yc)
    for mbin in (1, 50, 700, 2047):
        w = 2 * math.pi * mbin / (n * dbar)
        A = of.dft_power(y, np.array([w]), dbar)[0]
        assert abs(A - abs(F[mbin]) ** 2 / (n * np.mean(yc * yc))) <= 1e-9 * A


def test_features_structure():
    """Bins are the averages of four sub-frequencies spread over the bin;
    the top sub-frequency stays below the Nyquist frequency pi / dbar; the
    grid is the mean spacing (times only enter through it)."""
    w = of.sub_frequencies()
    assert w.shape == (64, 4) and np.all(np.diff(w.ravel()) > 0)
    assert w.max() < math.pi / 0.01
    rng = np.random.default_rng(8)
    t = np.cumsum(rng.exponential(0.01, 2000))
    y = rng.normal(size=2000)
    f = of.features(t, y)
    dbar = (t[-1] - t[0]) / 1999
    A = of.dft_power(y, w, dbar)
    assert np.allclose(f[:64], np.log(A.mean(axis=1) + 1e-8), rtol=0, atol=1e-12)
    t2 = np.linspace(t[0], t[-1], 2000)          # same mean spacing, other times
    assert np.allclose(of.features(t2, y), f, rtol=0, atol=1e-12)


def test_features_invariances_and_edge_cases():
    rng = np.random.default_rng(2)
    t = np.cumsum(rng.exponential(0.01, 3000))
    y = rng.normal(size=3000)
    f = of.features(t, y)
    g = of.features(t, 3.0 * y + 5.0)
    assert np.allclose(f[:64], g[:64], atol=1e-10)
    assert abs(g[64] - f[64] - math.log(9.0)) < 1e-12
    assert np.all(of.features(t, np.ones(3000)) == 0.0)
    assert np.all(of.features(t[:1], y[:1]) == 0.0)
    # white noise: the normalised periodogram averages to 1 over the bins
    assert abs(np.mean(np.exp(f[:64])) - 1.0) < 0.2


def test_noise_shows_as_the_high_frequency_plateau():
    """A smooth signal plus white noise of variance R on the Poisson grid:
    the top bins sit near R / (s2_signal + R) (the noise's share of the
    normalised periodogram), the low bins far above it."""
    rng = np.random.default_rng(9)
    n = 4096
    t = np.cumsum(rng.exponential(0.01, n))
    sig = np.sin(0.7 * t) + 0.5 * np.sin(1.9 * t)
    R = 0.01
    y = sig + rng.normal(0, math.sqrt(R), n)
    f = of.features(t, y)
    share = R / (np.var(sig) + R)
    assert abs(np.mean(f[56:64]) - math.log(share)) < 0.5
    assert f[:8].max() > math.log(share) + 5


# ---------------------------------------------------------------------------
# the network oracle
# ---------------------------------------------------------------------------
from oracle import mlp as om_mlp  # noqa: E402


def _net_inputs(M=32, seed=3):
    rng = np.random.default_rng(seed)
    feat = rng.normal(size=(M, 65)).astype(np.float32)
    theta = rng.normal(size=(M, 3))
    norm = np.zeros(144)
    norm[:65] = rng.normal(0, 0.1, 65)
    norm[65:130] = rng.uniform(0.5, 2.0, 65)
    norm[130:133] = rng.normal(0, 0.2, 3)
    norm[133:136] = rng.uniform(0.5, 2.0, 3)
    return feat, theta, norm.astype(np.float32).astype(np.float64)


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(4).normal(size=20_000) * np.exp(np.random.default_rng(5).uniform(-20, 20, 20_000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om_mlp.bf16(x), ref)


def test_network_gradient_equals_autograd_and_differences():
    """Without the bfloat16 rounding the oracle's backward pass is the exact
    gradient: equal to torch autograd in float64 and to central differences."""
    import torch
    feat, theta, norm = _net_inputs()
    p = om_mlp.random_params(6)
    loss, g, out = om_mlp.loss_grad(p, norm, feat, theta, rounding=False)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    W1 = pt[om_mlp.OW1:om_mlp.OB1].reshape(256, 80)
    W2 = pt[om_mlp.OW2:om_mlp.OB2].reshape(256, 256)
    W3 = pt[om_mlp.OW3:om_mlp.OB3].reshape(16, 256)
    X = torch.zeros(32, 80, dtype=torch.float64)
    X[:, :65] = (torch.tensor(feat, dtype=torch.float64) - torch.tensor(norm[:65])) / torch.tensor(norm[65:130])
    H1 = torch.relu(X @ W1.T + pt[om_mlp.OB1:om_mlp.OW2])
    H2 = torch.relu(H1 @ W2.T + pt[om_mlp.OB2:om_mlp.OW3])
    o = H2 @ W3.T + pt[om_mlp.OB3:]
    tn = (torch.tensor(theta) - torch.tensor(norm[130:133])) / torch.tensor(norm[133:136])
    lt = 0.5 * ((o[:, :3] - tn) ** 2).sum() / 32
    lt.backward()
    assert abs(lt.item() - loss) < 1e-13 * abs(loss)
    assert np.allclose(pt.grad.numpy(), g, rtol=1e-10, atol=1e-14)
    rng = np.random.default_rng(7)
    for i in rng.choice(np.flatnonzero(g != 0.0), 12, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (om_mlp.loss_grad(pp, norm, feat, theta, rounding=False)[0]
              - om_mlp.loss_grad(pm, norm, feat, theta, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3)
