"""Oracle of the learned initialisation's inputs: the 64-bin log periodogram
and the log sample variance of a series (65 features).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition (the learned-initialisation workload: a small network proposes
initial hyperparameters of the marginal-likelihood fit of Sec. 2 from a
log-periodogram of the series).  For a series y_k, k < n (n >= 2), with
mean ybar, variance s2 = sum (y_k - ybar)^2 / n and mean spacing
dbar = (t_{n-1} - t_0) / (n - 1), the periodogram is taken on the regular
grid k dbar (on the Poisson time grid of the workload, a smooth signal then
stays smooth from sample to sample and the measurement noise shows as the
high-frequency plateau; at the true times the random sampling would leak the
signal's power into a white floor that hides the noise):

    A(w) = |sum_k (y_k - ybar) exp(-i w k dbar)|^2 / (n s2),
    P_j  = 1/4 sum_{q<4} A(w_lo r^(j + (q - 3/2) / 4)),   j < 64,
    r    = (w_hi / w_lo)^(1 / 63),  w_lo = 2 pi / 40.96,  w_hi = 0.9 pi / 0.01,

(each bin averages four sub-frequencies spread over its width in log
frequency), features log(P_j + 1e-8), j < 64, and log(s2).  A series with
n < 2 or s2 = 0 gives zeros.
"""
from __future__ import annotations

import math

import numpy as np

NFREQ = 64
NSUB = 4
W_LO = 2.0 * math.pi / 40.96
W_HI = 0.9 * math.pi / 0.01


def sub_frequencies() -> np.ndarray:
    """[64, 4] angular frequencies (per unit time at spacing dbar)."""
    r = (W_HI / W_LO) ** (1.0 / (NFREQ - 1))
    e = np.arange(NFREQ)[:, None] + (np.arange(NSUB)[None, :] - 1.5) / NSUB
    return W_LO * r ** e


def dft_power(y: np.ndarray, w: np.ndarray, dbar: float) -> np.ndarray:
    """A(w) for the given frequencies, by direct sums (float64)."""
    n = y.size
    yc = y - y.mean()
    s2 = float(np.mean(yc * yc))
    ph = np.outer(np.ravel(w), np.arange(n) * dbar)
    re = np.cos(ph) @ yc
    im = -np.sin(ph) @ yc
    return ((re * re + im * im) / (n * s2)).reshape(np.shape(w))


def features(t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The 65 features of one series."""
    n = y.size
    out = np.zeros(NFREQ + 1)
    if n < 2:
        return out
    s2 = float(np.mean((y - y.mean()) ** 2))
    if not s2 > 0.0:
        return out
    dbar = (t[-1] - t[0]) / (n - 1)
    P = dft_power(y, sub_frequencies(), dbar).mean(axis=1)
    out[:NFREQ] = np.log(P + 1e-8)
    out[NFREQ] = math.log(s2)
    return out
