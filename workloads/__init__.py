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
