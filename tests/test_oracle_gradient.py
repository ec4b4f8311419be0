"""Pins of the oracle's log-likelihood gradient (forward mode) with respect to
theta = (log lengthscale, log variance, log noise variance).

The forward-mode oracle differentiates the discretisation (Frechet derivative
of the Van Loan exponential) and every line of the sequential Kalman filter.
It is pinned against things it shares no code with:

* the dense GP gradient 1/2 a^T dK a - 1/2 tr(K^-1 dK) (Sec. 2, parameter
  estimation; supplement Lemma) with the textbook Matern covariance and its
  lengthscale derivative written out by hand;
* central finite differences of the oracle's own log-likelihood, rebuilding
  the model at the shifted hyperparameters (also for the RBF Taylor model,
  which has no closed-form covariance);
* closed forms: far-apart observations (independent N(0, s2 + R) terms), an
  all-missing series (zero), the noise derivative of a one-point series;
* planted mistakes in a copy of the tangent code are caught.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense_gp
from oracle import model as om
import workloads as wl

NU = {"matern12": 0.5, "matern32": 1.5, "matern52": 2.5}


def dense_grad(kind, ell, s2, t, y, mask, R):
    nu = NU[kind]
    k = om.matern_kernel(nu, ell, s2)
    dk = om.matern_kernel_dlogl(nu, ell, s2)
    obs = mask.astype(bool)
    ll, g = dense_gp.loglik_grad(k, [dk, k, None], t[obs], y[obs], R, R)
    return ll, np.array(g)


def rel(a, b, n):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), n))


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52"])
def test_forward_mode_equals_dense_gp_gradient(kind):
    s = wl.sinusoid_small()
    t, y = s.t_train[:600], s.y_train[:600]
    rng = np.random.default_rng(3)
    mask = (rng.uniform(size=t.size) > 0.15).astype(np.uint8)
    for ell, s2, R in [(0.5, 1.0, 0.01), (2.0, 0.4, 0.1), (0.07, 3.0, 0.003)]:
        ll, g = oracle.loglik_grad_fwd(kind, ell, s2, t, y, mask, R)
        lld, gd = dense_grad(kind, ell, s2, t, y, mask, R)
        assert abs(ll - lld) <= 1e-10 * max(abs(lld), t.size)
        assert rel(g, gd, mask.sum()) <= 1e-10, (kind, ell, g, gd)


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_forward_mode_equals_central_differences(kind):
    s = wl.prefix(wl.sinusoid_large(N=1 << 14, M=100), 1500)
    t, y = s.t_train, s.y_train
    mask = np.ones(t.size, np.uint8)
    mask[100:180] = 0                      # a run of missing steps
    t = t.copy(); t[800:] += 7.0           # a long gap (doubling path)
    ll, g = oracle.loglik_grad_fwd(kind, 1.3, 0.8, t, y, mask, 0.02)
    gfd = oracle.loglik_grad_fd(kind, 1.3, 0.8, t, y, mask, 0.02)
    assert rel(g, gfd, mask.sum()) <= 1e-8, (g, gfd)


def test_per_step_noise_derivative_scales_every_R():
    s = wl.sinusoid_small()
    t, y = s.t_train[:300], s.y_train[:300]
    mask = np.ones(t.size, np.uint8)
    R = np.exp(np.random.default_rng(4).uniform(np.log(1e-3), np.log(1e-1), t.size))
    ll, g = oracle.loglik_grad_fwd("matern52", 0.6, 1.1, t, y, mask, R)
    gfd = oracle.loglik_grad_fd("matern52", 0.6, 1.1, t, y, mask, R)
    assert rel(g, gfd, t.size) <= 1e-8


def test_far_apart_observations_closed_form():
    """With steps >> lengthscale the observations are independent
    N(0, s2 + R): l = sum -1/2 [log 2 pi (s2 + R) + y^2 / (s2 + R)], so
    dl/dlog s2 = sum -1/2 s2 [1/(s2+R) - y^2/(s2+R)^2], the same with R for
    the noise, and dl/dlog l = 0 up to exp(-gap / l) terms."""
    rng = np.random.default_rng(5)
    n = 40
    t = np.arange(n) * 400.0
    y = rng.normal(0, 1.2, n)
    mask = np.ones(n, np.uint8)
    s2, R = 1.7, 0.3
    for kind in ("matern32", "matern52", "rbf"):
        ll, g = oracle.loglik_grad_fwd(kind, 1.0, s2, t, y, mask, R)
        # prior variance of f: s2 for Matern; H P_inf H^T (proportional to s2)
        # for the RBF Taylor model
        m = om.make_model(kind, 1.0, s2)
        v0 = (m.H @ m.Pinf @ m.H.T).item()
        V = v0 + R
        gs = np.sum(-0.5 * v0 * (1.0 / V - y * y / V ** 2))
        gr = np.sum(-0.5 * R * (1.0 / V - y * y / V ** 2))
        assert abs(g[1] - gs) <= 1e-12 * n and abs(g[2] - gr) <= 1e-12 * n
        assert abs(g[0]) <= 1e-12 * n


def test_all_missing_gradient_is_zero():
    t = np.linspace(0, 5, 50)
    ll, g = oracle.loglik_grad_fwd("matern52", 0.8, 1.0, t, np.zeros(50), np.zeros(50, np.uint8), 0.01)
    assert ll == 0.0 and np.all(g == 0.0)


def test_single_point_noise_derivative():
    """n = 1: l = -1/2 [log 2 pi (s2 + R) + y^2/(s2 + R)] in closed form."""
    for kind in ("matern12", "matern32", "matern52"):
        y0, s2, R = 0.7, 1.4, 0.2
        ll, g = oracle.loglik_grad_fwd(kind, 0.3, s2, np.array([2.0]), np.array([y0]), np.ones(1, np.uint8), R)
        V = s2 + R
        assert abs(ll + 0.5 * (math.log(2 * math.pi * V) + y0 * y0 / V)) < 1e-15
        assert abs(g[1] + 0.5 * s2 * (1 / V - y0 * y0 / V ** 2)) < 1e-15
        assert abs(g[2] + 0.5 * R * (1 / V - y0 * y0 / V ** 2)) < 1e-15
        assert abs(g[0]) < 1e-14          # H P_inf H^T = s2 does not depend on l


# ---------------------------------------------------------------------------
# planted mistakes in the tangent code
# ---------------------------------------------------------------------------
SRC = os.path.join(os.path.dirname(oracle.__file__), "ssgp_oracle.c")

MUTANTS = [
    ("drop_dF_P_Ft", "mm(d, d, d, dF, P, T); mm(d, d, d, T, Ft, A);\n    for (int i = 0; i < dd; ++i) dPp[i] += A[i];",
     "mm(d, d, d, dF, P, T); mm(d, d, d, T, Ft, A);"),
    ("tangent_dv_sign", "dv -= H[i] * dmp[i];", "dv += H[i] * dmp[i];"),
    ("tangent_dK_no_dS", "dK[i] = (dPH[i] - K[i] * dS) / S;", "dK[i] = dPH[i] / S;"),
    ("tangent_dll_drops_term", " - v * v * dS / (S * S));", ");"),
    ("tangent_dm_drops_dK", "dm[i] = dmp[i] + dK[i] * v + K[i] * dv;", "dm[i] = dmp[i] + K[i] * dv;"),
    ("frechet_drops_dE12", "dQ[i] = T1[i] + T2[i];  /* dQ", "dQ[i] = T1[i];  /* dQ"),
    ("frechet_dW_sign", "X[i * N + n + d + j] = dW[i * d + j] * h;", "X[i * N + n + d + j] = -dW[i * d + j] * h;"),
    ("frechet_dF_untransposed", "dF[i * d + j] = E[(d + j) * N + n + d + i];",
     "dF[i * d + j] = E[(d + i) * N + n + d + j];"),
    ("doubling_dF_one_sided", "for (int i = 0; i < d * d; ++i) dF[i] = A1[i] + A2[i];",
     "for (int i = 0; i < d * d; ++i) dF[i] = 2.0L * A2[i];"),
    ("doubling_dQ_drops_cross", "dQ[i] += A1[i] + A2[i] + A3[i];", "dQ[i] += A2[i];"),
    ("first_step_dPinf_dropped", "dQ_[i] = dPinf_[i];", "dQ_[i] = 0.0;"),
]


def _battery():
    rng = np.random.default_rng(22)
    n = 150
    t = np.sort(rng.uniform(0, 12, n))
    t[100:] += 30.0                                  # one long step (doubling)
    mask = (rng.uniform(size=n) > 0.2).astype(np.uint8)
    y = np.sin(2 * t) + rng.normal(0, 0.1, n)
    for kind in ("matern32", "matern52"):
        ll, g = oracle.loglik_grad_fwd(kind, 0.7, 1.3, t, y, mask, 0.02)
        lld, gd = dense_grad(kind, 0.7, 1.3, t, y, mask, 0.02)
        assert rel(g, gd, mask.sum()) <= 1e-9, (kind, g, gd)


def _with_source(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / f"{name}.so"))
    oracle.use_library(lib)


def test_unmodified_gradient_oracle_passes_battery(tmp_path):
    try:
        _with_source(tmp_path, "control", open(SRC).read())
        _battery()
    finally:
        oracle.use_library(None)


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_gradient_mistake_is_caught(tmp_path, name, orig, bad):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    try:
        _with_source(tmp_path, name, text.replace(orig, bad, 1))
        with pytest.raises((AssertionError, RuntimeError, np.linalg.LinAlgError, ValueError)):
            _battery()
    finally:
        oracle.use_library(None)
