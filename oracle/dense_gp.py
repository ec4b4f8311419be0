"""Dense O(N^3) GP regression -- the quantity the state-space method reproduces.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The supplement's Lemma (equivalence of state-space GP and standard GP) and its
Corollary state that the (parallel) Kalman smoother recovers the GP posterior
mean and variance at every time point.  This module computes that posterior
directly with a Cholesky factorisation, together with the log marginal
likelihood log N(y; 0, K + R) of Sec. 2 (parameter estimation).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cho_factor, cho_solve


def posterior(kfun, t_all: np.ndarray, mask: np.ndarray, y_all: np.ndarray, R):
    """Posterior mean and variance of f at every t_all, given y at mask==1.
    R is a scalar noise variance or one per step (only observed ones used).

    Returns (mean, var, loglik)."""
    obs = mask.astype(bool)
    to = t_all[obs]
    yo = y_all[obs]
    R = np.asarray(R, dtype=np.float64)
    Ro = R[obs] if R.ndim == 1 and R.size == t_all.size else np.full(to.size, float(R))
    Koo = kfun(to[:, None] - to[None, :]) + np.diag(Ro)
    cf = cho_factor(Koo, lower=True)
    alpha = cho_solve(cf, yo)
    Kao = kfun(t_all[:, None] - to[None, :])
    mean = Kao @ alpha
    V = cho_solve(cf, Kao.T)
    var = kfun(np.zeros(1))[0] - np.einsum("ij,ji->i", Kao, V)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    loglik = -0.5 * float(yo @ alpha) - 0.5 * logdet - 0.5 * to.size * math.log(2.0 * math.pi)
    return mean, var, loglik


def loglik_grad(kfun, dkfuns, t: np.ndarray, y: np.ndarray, R: float, dR: float):
    """Gradient of log N(y; 0, K + R I) with respect to parameters theta_i,
    given dK/dtheta_i as covariance functions dkfuns[i] (None for the noise
    parameter, whose derivative is dR I):
        d loglik / d theta = 1/2 alpha^T dK alpha - 1/2 tr(K^-1 dK),
        alpha = (K + R I)^-1 y.
    Returns (loglik, [gradients])."""
    tau = t[:, None] - t[None, :]
    Ky = kfun(tau) + R * np.eye(t.size)
    cf = cho_factor(Ky, lower=True)
    alpha = cho_solve(cf, y)
    Kinv = cho_solve(cf, np.eye(t.size))
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    ll = -0.5 * float(y @ alpha) - 0.5 * logdet - 0.5 * t.size * math.log(2.0 * math.pi)
    out = []
    for dk in dkfuns:
        dK = dR * np.eye(t.size) if dk is None else dk(tau)
        out.append(0.5 * float(alpha @ dK @ alpha) - 0.5 * float(np.sum(Kinv * dK)))
    return ll, out
