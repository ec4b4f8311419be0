"""Pins for the oracle's discretisation, supplement Eq. (ss-gp-formation).

Checked against: the Ornstein-Uhlenbeck (Matern-1/2) closed form, a library
matrix exponential, stationarity F P_inf F^T + Q = P_inf (Sec. 4.1), the
Lyapunov identity G Q + Q G^T = F W F^T - W of the integral, and a
50-digit evaluation of Q by mpmath quadrature-free Van Loan (entrywise,
including entries that are many orders smaller than P_inf).
"""
import math

import mpmath
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle import model as om


def test_matern12_closed_form(oracle_lib):
    ell, s2 = 0.7, 1.9
    m = om.make_model("matern12", ell, s2)
    t = np.array([0.0, 1e-6, 1e-3, 0.5, 0.5, 3.0, 40.0])
    F, Q = oracle.discretize(m, t)
    for k in range(1, t.size):
        h = t[k] - t[k - 1]
        assert abs(F[k, 0, 0] - math.exp(-h / ell)) <= 1e-15
        q_ref = -s2 * math.expm1(-2 * h / ell)
        assert abs(Q[k, 0, 0] - q_ref) <= 1e-14 * max(q_ref, 1e-300) + 1e-300
    assert F[0, 0, 0] == 0.0 and Q[0, 0, 0] == pytest.approx(s2)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("balanced", [False, True])
def test_stationarity_and_expm(oracle_lib, kind, balanced):
    m = om.make_model(kind, 1.0, 1.0, balanced=balanced)
    t = np.cumsum([0.0, 1e-5, 1e-3, 0.02, 0.3, 2.0, 0.0, 9.0])
    F, Q = oracle.discretize(m, t)
    for k in range(1, t.size):
        h = t[k] - t[k - 1]
        np.testing.assert_allclose(F[k], expm(m.G * h), rtol=0, atol=1e-13 * max(1.0, np.abs(F[k]).max()))
        lhs = F[k] @ m.Pinf @ F[k].T + Q[k]
        assert np.max(np.abs(lhs - m.Pinf)) <= 1e-13 * np.max(np.abs(m.Pinf))
        np.testing.assert_array_equal(Q[k], Q[k].T)
        ev = np.linalg.eigvalsh(Q[k])
        assert ev.min() >= -1e-14 * max(ev.max(), 1e-300)
    # h = 0 (duplicate time): F = I, Q = 0 exactly
    np.testing.assert_array_equal(F[6], np.eye(m.d))
    np.testing.assert_array_equal(Q[6], np.zeros((m.d, m.d)))


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("balanced", [False, True])
def test_lyapunov_identity_of_the_integral(oracle_lib, kind, balanced):
    """d/dh of Q(h) = int_0^h e^{sG} W e^{sG}^T ds is G Q + Q G^T + W and also
    F W F^T, so G Q + Q G^T = F W F^T - W at every step (the identity from
    which the device forms rows 1..d-1 of Q).  Checked against the scale of
    its terms, over steps from 1e-4 to 10 lengthscales."""
    m = om.make_model(kind, 1.0, 1.0, balanced=balanced)
    h = np.array([1e-4, 3e-3, 0.05, 0.4, 2.0, 10.0])
    t = np.cumsum(np.concatenate([[0.0], h]))
    F, Q = oracle.discretize(m, t)
    W = m.W
    for k in range(1, t.size):
        lhs = m.G @ Q[k] + Q[k] @ m.G.T
        rhs = F[k] @ W @ F[k].T - W
        scale = np.abs(m.G).max() * np.abs(Q[k]).max() + np.abs(W).max()
        assert np.abs(lhs - rhs).max() <= 1e-13 * scale, (k, np.abs(lhs - rhs).max() / scale)


def _mp_vanloan(G, W, h, dps=50):
    mpmath.mp.dps = dps
    d = G.shape[0]
    C = mpmath.zeros(2 * d, 2 * d)
    for i in range(d):
        for j in range(d):
            C[i, j] = -mpmath.mpf(G[i, j]) * mpmath.mpf(h)
            C[i, d + j] = mpmath.mpf(W[i, j]) * mpmath.mpf(h)
            C[d + i, d + j] = mpmath.mpf(G[j, i]) * mpmath.mpf(h)
    E = mpmath.expm(C)
    F = mpmath.matrix(d, d); E12 = mpmath.matrix(d, d)
    for i in range(d):
        for j in range(d):
            F[i, j] = E[d + j, d + i]
            E12[i, j] = E[i, d + j]
    Q = F * E12
    return np.array(F.tolist(), dtype=float), np.array(Q.tolist(), dtype=float)


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
@pytest.mark.parametrize("h", [1e-3, 0.05])
def test_entrywise_accuracy_small_steps(oracle_lib, kind, h):
    """Compared with a 50-digit evaluation: Q is accurate to 1e-17 of its
    largest entry everywhere, and entrywise to 1e-13 on every entry larger
    than 1e-12 of the largest (the order-6 RBF spans 30 decades at h = 1e-3;
    the smallest entries, ~h^11, cannot influence any output); F entrywise."""
    m = om.make_model(kind, 1.0, 1.0, balanced=True)
    F, Q = oracle.discretize(m, np.array([0.0, h]))
    Fr, Qr = _mp_vanloan(m.G, m.W, h)
    qmax = np.abs(Qr).max()
    assert np.abs(Q[1] - Qr).max() <= 1e-17 * qmax
    big = np.abs(Qr) >= 1e-12 * qmax
    rel = np.abs(Q[1][big] - Qr[big]) / np.abs(Qr[big])
    assert rel.max() <= 1e-13, rel.max()
    relF = np.abs(F[1] - Fr) / np.maximum(np.abs(Fr), 1e-300)
    assert relF.max() <= 1e-14


def test_unsorted_times_rejected(oracle_lib):
    m = om.make_model("matern32", 1.0, 1.0)
    with pytest.raises(RuntimeError):
        oracle.discretize(m, np.array([0.0, 1.0, 0.5]))
