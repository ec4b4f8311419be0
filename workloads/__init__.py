"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the method's arithmetic: it only draws times and
noisy sinusoids (the paper's simulated workload, Sec. 5.1: noisy sums of
sinusoids observed at sorted times) with numpy's PCG64 generator.  Both the
oracle and the CUDA path consume exactly these arrays.

Workloads (hyperparameters are passed separately):

* ``sinusoid_small`` -- 1,000 training times uniform on [0, 10] (sorted),
  y = sin(2 pi t) + sin(5 pi t) + N(0, 0.1^2), plus 100 prediction times
  uniform on [0, 10].  Matern-3/2, lengthscale 0.5, variance 1, noise 0.01.
* ``sinusoid_large`` -- 2^20 training times uniform on [0, 1000],
  y = sin(0.3 t) + 0.5 sin(1.7 t) + N(0, 0.1^2), plus 10,000 prediction
  times uniform on [0, 1000].  RBF (Taylor order 6, d = 6) and Matern-5/2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Series:
    t_train: np.ndarray
    y_train: np.ndarray
    t_test: np.ndarray

    @property
    def N(self) -> int:
        return self.t_train.size

    @property
    def M(self) -> int:
        return self.t_test.size


def sinusoid_small(seed: int = 1, N: int = 1000, M: int = 100) -> Series:
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 10.0, N))
    y = np.sin(2.0 * np.pi * t) + np.sin(5.0 * np.pi * t) + rng.normal(0.0, 0.1, N)
    ts = np.sort(rng.uniform(0.0, 10.0, M))
    return Series(t, y, ts)


def sinusoid_large(seed: int = 2, N: int = 1 << 20, M: int = 10_000, T: float = 1000.0) -> Series:
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, T, N))
    y = np.sin(0.3 * t) + 0.5 * np.sin(1.7 * t) + rng.normal(0.0, 0.1, N)
    ts = np.sort(rng.uniform(0.0, T, M))
    return Series(t, y, ts)


def prefix(s: Series, n_train: int) -> Series:
    """The first n_train training points and the prediction points inside
    their time span (a small slice of a large workload, same spacing)."""
    t = s.t_train[:n_train]
    y = s.y_train[:n_train]
    ts = s.t_test[s.t_test <= t[-1]]
    return Series(t.copy(), y.copy(), ts.copy())


def random_series(seed: int, N: int, M: int, T: float, noise: float = 0.1) -> Series:
    """Generic noisy sinusoid on [0, T] for edge-case sweeps."""
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, T, N))
    y = np.sin(0.3 * t) + 0.5 * np.sin(1.7 * t) + rng.normal(0.0, noise, N)
    ts = np.sort(rng.uniform(0.0, T, M))
    return Series(t, y, ts)


# Hyperparameters of the workloads (the large workload's are not fixed by the
# paper; lengthscale 1, variance 1, noise variance 0.01 are this build's reading).
SMALL = dict(kind="matern32", lengthscale=0.5, variance=1.0, noise=0.01)
LARGE_RBF = dict(kind="rbf", order=6, lengthscale=1.0, variance=1.0, noise=0.01)
LARGE_M52 = dict(kind="matern52", lengthscale=1.0, variance=1.0, noise=0.01)


@dataclass
class Batch:
    """B independent series concatenated: series s is t[offsets[s]:offsets[s+1]]."""
    t: np.ndarray
    y: np.ndarray
    offsets: np.ndarray      # int64[B + 1]
    kind: list               # kernel family per series ("matern32" / "matern52")
    lengthscale: np.ndarray
    variance: np.ndarray
    noise: np.ndarray        # noise variance R per series

    @property
    def B(self) -> int:
        return self.offsets.size - 1

    def params(self, idx=None) -> np.ndarray:
        """(lengthscale, variance, noise) rows, float64[B, 3] (or the rows idx)."""
        p = np.stack([self.lengthscale, self.variance, self.noise], axis=1)
        return p if idx is None else p[idx]

    def series(self, s: int):
        a, b = self.offsets[s], self.offsets[s + 1]
        return self.t[a:b], self.y[a:b]


def series_batch(seed: int = 3, B: int = 4096, n_min: int = 1000, n_max: int = 65536, spacing: float = 0.01,
                 kinds=("matern32", "matern52"), lengths=None) -> Batch:
    """Many independent series of uneven length (the batched hyperparameter
    search workload): lengths log-uniform on [n_min, n_max] (or given),
    times sorted uniform on [0, spacing * n], kernel family drawn uniformly
    from `kinds`, lengthscale log-uniform on [0.1, 10], variance 1, noise
    variance log-uniform on [1e-3, 1e-1].  y is a random two-tone sinusoid at
    frequencies set by the series' lengthscale, with N(0, R) noise."""
    rng = np.random.default_rng(seed)
    if lengths is None:
        lengths = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), B))).astype(np.int64)
    lengths = np.asarray(lengths, dtype=np.int64)
    B = lengths.size
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    kind = [kinds[i] for i in rng.integers(0, len(kinds), B)]
    ell = np.exp(rng.uniform(np.log(0.1), np.log(10.0), B))
    var = np.ones(B)
    R = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), B))
    n = int(offsets[-1])
    t = np.empty(n)
    y = np.empty(n)
    for s in range(B):
        a, b = offsets[s], offsets[s + 1]
        m = b - a
        ts = np.sort(rng.uniform(0.0, spacing * m, m))
        w1, w2 = rng.uniform(0.5, 2.0, 2) / ell[s]
        ph = rng.uniform(0.0, 2.0 * np.pi, 2)
        t[a:b] = ts
        y[a:b] = np.sin(w1 * ts + ph[0]) + 0.5 * np.sin(w2 * ts + ph[1]) + rng.normal(0.0, np.sqrt(R[s]), m)
    return Batch(t, y, offsets, kind, ell, var, R)


def subset(bt: Batch, idx) -> Batch:
    """The series idx of a batch, re-concatenated in that order."""
    idx = np.asarray(idx, dtype=np.int64)
    lengths = bt.offsets[idx + 1] - bt.offsets[idx]
    offsets = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    t = np.concatenate([bt.t[bt.offsets[s]:bt.offsets[s + 1]] for s in idx]) if idx.size else np.empty(0)
    y = np.concatenate([bt.y[bt.offsets[s]:bt.offsets[s + 1]] for s in idx]) if idx.size else np.empty(0)
    return Batch(t, y, offsets, [bt.kind[s] for s in idx], bt.lengthscale[idx].copy(), bt.variance[idx].copy(),
                 bt.noise[idx].copy())


BATCH = dict(seed=3, B=4096, n_min=1000, n_max=65536, spacing=0.01)


def prior_spec(seed: int, B: int, n: int | None = None, n_min: int | None = None, n_max: int | None = None,
               ell=(0.1, 10.0), var=(0.1, 10.0), noise=(1e-3, 1e-1)):
    """Lengths and hyperparameters of B series to be drawn from a prior:
    (lengthscale, variance, noise variance) each log-uniform on its range;
    lengths all n, or log-uniform on [n_min, n_max].  Returns
    (offsets int64[B+1], params float64[B, 3])."""
    rng = np.random.default_rng(seed)
    if n is not None:
        lengths = np.full(B, int(n), dtype=np.int64)
    else:
        lengths = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), B))).astype(np.int64)
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    lo = np.log([ell[0], var[0], noise[0]])
    hi = np.log([ell[1], var[1], noise[1]])
    params = np.exp(rng.uniform(lo, hi, (B, 3)))
    return offsets, params


def prior_batch_spec(seed: int = 3, B: int = 4096, n_min: int = 1000, n_max: int = 65536):
    """The batched workload with its y drawn from the state-space prior: per
    series the length (log-uniform on [n_min, n_max]), the kernel family
    (Matern-3/2 or 5/2, each with probability 1/2) and (lengthscale, variance,
    noise variance) = (log-uniform [0.1, 10], 1, log-uniform [1e-3, 1e-1]).
    The times and y are drawn by a prior simulation (Poisson time grid of mean
    spacing 0.01), which this module does not do.  Returns (offsets
    int64[B+1], kinds list[B], params float64[B, 3])."""
    rng = np.random.default_rng(seed)
    lengths = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), B))).astype(np.int64)
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    kinds = [("matern32", "matern52")[i] for i in rng.integers(0, 2, B)]
    params = np.stack([np.exp(rng.uniform(np.log(0.1), np.log(10.0), B)), np.ones(B),
                       np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), B))], axis=1)
    return offsets, kinds, params


PRIOR_BATCH = dict(seed=3, B=4096, n_min=1000, n_max=65536)


def subset_spec(offsets: np.ndarray, params: np.ndarray, idx):
    """Offsets and parameter rows of the series idx, re-concatenated in that order."""
    idx = np.asarray(idx, dtype=np.int64)
    lengths = offsets[idx + 1] - offsets[idx]
    off = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off, params[idx].copy()


# The learned-initialisation workload: Matern-5/2 prior series, mean spacing
# 0.01 (a Poisson time grid), log-uniform hyperparameters.
LEARN_TRAIN = dict(seed=50, B=1_000_000, n=4096)
LEARN_HELDOUT = dict(seed=51, B=4096, n_min=4096, n_max=65536)


def sunspot_like(seed: int = 7, N: int = 3200, M: int = 96_000) -> Series:
    """Shape-only stand-in for the paper's monthly sunspot series (Sec. 5.2:
    N = 3,200 monthly training points, 96,000 daily prediction times): times
    in years, monthly training times (k + 1/2) / 12, daily prediction times
    (j + 1/2) / 365.25, and an 11-year quasi-periodic non-negative signal
    80 |sin(pi t / 11)|^1.5 (1 + 0.3 sin(2 pi t / 90)) with N(0, 15^2) noise.
    No sunspot data is reproduced."""
    rng = np.random.default_rng(seed)
    t = (np.arange(N) + 0.5) / 12.0
    sig = 80.0 * np.abs(np.sin(np.pi * t / 11.0)) ** 1.5 * (1.0 + 0.3 * np.sin(2.0 * np.pi * t / 90.0))
    y = sig + rng.normal(0.0, 15.0, N)
    ts = (np.arange(M) + 0.5) / 365.25
    return Series(t, y, ts)
