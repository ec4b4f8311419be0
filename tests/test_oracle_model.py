"""Pins for the oracle's model formation (Sec. 2, Sec. 4.1, Sec. 4.2).

Each check compares against something other than the oracle itself: textbook
Matern covariances, the Taylor-approximated RBF spectral density evaluated
directly, a library matrix exponential, and the Lyapunov residual.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import model as om

KINDS = [("matern12", 0.5), ("matern32", 1.5), ("matern52", 2.5)]


@pytest.mark.parametrize("kind,nu", KINDS)
@pytest.mark.parametrize("ell,s2", [(0.5, 1.0), (1.0, 2.0), (7.0, 0.3)])
def test_matern_sde_reproduces_textbook_covariance(kind, nu, ell, s2):
    """H exp(G tau) P_inf H^T equals the textbook Matern covariance (Sec. 2:
    the Matern state-space form is exact)."""
    m = om.make_model(kind, ell, s2)
    k = om.matern_kernel(nu, ell, s2)
    for tau in [0.0, 0.01 * ell, 0.3 * ell, ell, 2.5 * ell, 6.0 * ell]:
        c = (m.H @ expm(m.G * tau) @ m.Pinf @ m.H.T)[0, 0]
        assert abs(c - k(tau)) <= 1e-12 * s2, (tau, c, k(tau))


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
@pytest.mark.parametrize("ell", [0.1, 1.0, 10.0])
def test_lyapunov_residual(kind, ell):
    """G P_inf + P_inf G^T + L q L^T = 0 (Sec. 4.1)."""
    m = om.make_model(kind, ell, 1.0)
    res = m.G @ m.Pinf + m.Pinf @ m.G.T + m.W
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(m.W))
    np.testing.assert_array_equal(m.Pinf, m.Pinf.T)
    assert np.all(np.linalg.eigvalsh(m.Pinf) > 0)


def test_matern32_pinf_closed_form():
    ell, s2 = 0.7, 1.3
    lam = math.sqrt(3) / ell
    m = om.make_model("matern32", ell, s2)
    np.testing.assert_allclose(m.Pinf, np.diag([s2, lam * lam * s2]), rtol=1e-13, atol=1e-13 * s2)


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("ell,s2", [(1.0, 1.0), (0.3, 2.0)])
def test_rbf_taylor_spectral_density(order, ell, s2):
    """q |H (i w - G)^{-1} L|^2 equals the order-n Taylor approximation of the
    RBF spectral density, s2 sqrt(2 pi) l / sum_k (l^2 w^2/2)^k / k!."""
    m = om.make_model("rbf", ell, s2, order=order)
    for w in [0.0, 0.3 / ell, 1.0 / ell, 2.0 / ell, 5.0 / ell]:
        tf = m.H @ np.linalg.solve(1j * w * np.eye(m.d) - m.G, m.L)
        S_ssm = m.q * abs(tf[0, 0]) ** 2
        x = 0.5 * ell * ell * w * w
        S_tay = s2 * math.sqrt(2 * math.pi) * ell / sum(x ** k / math.factorial(k) for k in range(order + 1))
        assert abs(S_ssm - S_tay) <= 1e-10 * S_tay, (w, S_ssm, S_tay)


@pytest.mark.parametrize("ell", [0.2, 1.0, 5.0])
def test_rbf_taylor_is_stable_and_close_to_rbf(ell):
    """The factor is Hurwitz; the order-6 model is within 1e-2 of the exact RBF
    covariance (the approximation of Sec. 2 is reported, not gated tightly)."""
    m = om.make_model("rbf", ell, 1.0)
    assert np.all(np.linalg.eigvals(m.G).real < 0)
    k = om.ssm_kernel(m)
    tau = np.linspace(0, 5 * ell, 41)
    exact = np.exp(-0.5 * (tau / ell) ** 2)
    assert np.max(np.abs(k(tau) - exact)) < 1e-2
    assert abs(m.Pinf[0, 0] - 1.0) < 1e-2


@pytest.mark.parametrize("order", [4, 6])
def test_ssm_kernel_eig_vs_expm(order):
    m = om.make_model("rbf", 0.8, 1.5, order=order)
    k = om.ssm_kernel(m)
    for tau in [0.0, 0.05, 0.4, 1.7, 4.0]:
        ref = (m.H @ expm(m.G * tau) @ m.Pinf @ m.H.T)[0, 0]
        assert abs(k(np.array([tau]))[0] - ref) <= 1e-9 * 1.5
    with pytest.raises(ValueError):
        om.ssm_kernel(om.make_model("matern52", 1.0, 1.0))


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_balancing_is_exact_similarity(kind):
    """Balanced model (Sec. 4.2): D powers of two with D_0 = 1, G' = D^{-1} G D,
    the stationary covariance transforms as D^{-1} P_inf D^{-1}, and the
    output covariance H' exp(G' tau) P_inf' H'^T is unchanged."""
    m = om.make_model(kind, 1.0, 1.0)
    b = om.make_model(kind, 1.0, 1.0, balanced=True)
    D = b.D
    assert D[0] == 1.0
    assert np.all(np.log2(D) == np.round(np.log2(D)))
    np.testing.assert_array_equal(b.G, np.diag(1 / D) @ m.G @ np.diag(D))
    res = b.G @ b.Pinf + b.Pinf @ b.G.T + b.W
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(b.W))
    for tau in [0.0, 0.3, 1.1]:
        c0 = (m.H @ expm(m.G * tau) @ m.Pinf @ m.H.T)[0, 0]
        c1 = (b.H @ expm(b.G * tau) @ b.Pinf @ b.H.T)[0, 0]
        assert abs(c0 - c1) <= 1e-12

    def spread(G):
        off = G - np.diag(np.diag(G))
        r = np.linalg.norm(off, axis=1); c = np.linalg.norm(off, axis=0)
        return np.max(np.maximum(r, c) / np.minimum(r, c))
    assert spread(b.G) <= spread(m.G)
