"""Oracle of the learned initialisation's inputs: the 64-bin log periodogram
and the log sample variance of a series (65 features).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition (the learned-initialisation workload: a small network proposes
initial hyperparameters of the marginal-likelihood fit of Sec. 2 from a
log-periodogram of the series): for a series (t_k, y_k), k < n, with mean ybar
and variance s2 = sum (y_k - ybar)^2 / n,
    P_j = |sum_k (y_k - ybar) exp(-i w_j (t_k - t_0))|^2 / (n s2),  j < 64,
at the angular frequencies w_j = w_lo (w_hi / w_lo)^(j / 63), w_lo = 2 pi / 40.96
(one period over 4096 steps of mean spacing 0.01), w_hi = pi / 0.01 (the
Nyquist frequency of the mean spacing).  Features: log(P_j + 1e-8), j < 64,
and log(s2).  A constant series (s2 = 0) gives zeros.
"""
from __future__ import annotations

import math

import numpy as np

NFREQ = 64
W_LO = 2.0 * math.pi / 40.96
W_HI = math.pi / 0.01


def frequencies() -> np.ndarray:
    return W_LO * (W_HI / W_LO) ** (np.arange(NFREQ) / (NFREQ - 1))


def features(t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The 65 features of one series, by the direct sums (float64)."""
    n = y.size
    out = np.zeros(NFREQ + 1)
    if n == 0:
        return out
    yc = y - y.mean()
    s2 = float(np.mean(yc * yc))
    if not s2 > 0.0:
        return out
    w = frequencies()
    ph = np.outer(w, t - t[0])
    re = np.cos(ph) @ yc
    im = -np.sin(ph) @ yc
    P = (re * re + im * im) / (n * s2)
    out[:NFREQ] = np.log(P + 1e-8)
    out[NFREQ] = math.log(s2)
    return out
