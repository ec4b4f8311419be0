"""Pins for the oracle's filter, smoother, log-likelihood, operators and merge.

Against: dense Cholesky GP regression (supplement Lemma + Corollary), closed
forms (one observation, far-apart observations, all missing), invariants
(symmetry, PSD, smoothed <= filtered <= prior variance, balancing), the
sequential-vs-parallel identities of Props. 1 and 2 (folds of the oracle's
own operators, random bracketings, all bracketings of small sequences), the
segment reset of the operators, and a brute-force merge.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import dense_gp
from oracle import model as om

NU = {"matern12": 0.5, "matern32": 1.5, "matern52": 2.5}


def rel_errors(f_mean, f_var, ll, mean, var, ll_ref, n_obs):
    """Tolerance semantics: mean relative to max(|m|, sqrt(v)), variance
    relative to v, log-likelihood relative to max(|l|, n_obs)."""
    em = np.max(np.abs(f_mean - mean) / np.maximum(np.abs(mean), np.sqrt(var)))
    ev = np.max(np.abs(f_var - var) / var)
    el = abs(ll - ll_ref) / max(abs(ll_ref), n_obs)
    return em, ev, el


def kernel_of(kind, m, ell, s2):
    return om.matern_kernel(NU[kind], ell, s2) if kind in NU else om.ssm_kernel(m)


def test_dense_gp_small_workload(oracle_lib):
    """The 1,000 + 100 point Matern-3/2 workload in full against dense GP."""
    s = wl.sinusoid_small()
    p = wl.SMALL
    m = om.make_model(p["kind"], p["lengthscale"], p["variance"])
    _, _, res, (t, y, mask, tp) = oracle.predict(m, s.t_train, s.y_train, s.t_test, p["noise"])
    mean, var, ll = dense_gp.posterior(kernel_of(p["kind"], m, 0.5, 1.0), t, mask, y, p["noise"])
    em, ev, el = rel_errors(res.f_mean, res.f_var, res.loglik, mean, var, ll, s.N)
    assert em < 1e-9 and ev < 1e-9 and el < 1e-9, (em, ev, el)


@pytest.mark.parametrize("kind,tol", [("matern52", 1e-9), ("rbf", 1e-6)])
@pytest.mark.parametrize("balanced", [False, True])
def test_dense_gp_large_workload_prefix(oracle_lib, kind, tol, balanced):
    """A 1,900-point prefix of the 2^20-point workload (same spacing)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 14, M=200), 1900)
    m = om.make_model(kind, 1.0, 1.0, balanced=balanced)
    _, _, res, (t, y, mask, tp) = oracle.predict(m, s.t_train, s.y_train, s.t_test, 0.01)
    mean, var, ll = dense_gp.posterior(kernel_of(kind, m, 1.0, 1.0), t, mask, y, 0.01)
    em, ev, el = rel_errors(res.f_mean, res.f_var, res.loglik, mean, var, ll, s.N)
    assert em < tol and ev < tol and el < tol, (em, ev, el)


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52"])
def test_dense_gp_heteroscedastic_and_ties(oracle_lib, kind):
    """Per-step noise variances (Eq. (gp-def): sigma_k^2) and duplicate times."""
    rng = np.random.default_rng(7)
    t = np.sort(np.concatenate([rng.uniform(0, 5, 60), [1.0, 1.0, 2.5]]))
    y = np.sin(t) + rng.normal(0, 0.1, t.size)
    mask = (rng.uniform(size=t.size) < 0.8).astype(np.uint8)
    R = rng.uniform(1e-3, 1e-1, t.size)
    m = om.make_model(kind, 0.8, 1.7)
    res = oracle.run(m, t, y * mask, mask, R)
    mean, var, ll = dense_gp.posterior(kernel_of(kind, m, 0.8, 1.7), t, mask, y * mask, R)
    em, ev, el = rel_errors(res.f_mean, res.f_var, res.loglik, mean, var, ll, int(mask.sum()))
    assert em < 1e-10 and ev < 1e-10 and el < 1e-12, (em, ev, el)


def test_single_observation_closed_form(oracle_lib):
    """N = 1: posterior f mean s2 y / (s2 + R), variance s2 - s2^2 / (s2 + R)."""
    s2, R, yv = 1.7, 0.2, 0.9
    for kind in ["matern32", "rbf"]:
        m = om.make_model(kind, 1.3, s2)
        res = oracle.run(m, np.array([2.0]), np.array([yv]), np.array([1], np.uint8), R)
        v0 = m.Pinf[0, 0]
        assert abs(res.f_mean[0] - v0 * yv / (v0 + R)) < 1e-15
        assert abs(res.f_var[0] - (v0 - v0 * v0 / (v0 + R))) < 1e-15
        ll = -0.5 * (math.log(2 * math.pi * (v0 + R)) + yv * yv / (v0 + R))
        assert abs(res.loglik - ll) < 1e-14


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_far_apart_observations_are_independent(oracle_lib, kind):
    """Gaps of 10^4 lengthscales: F -> 0, so the likelihood factorises into
    N(y_k; 0, P_inf_00 + R) and each posterior is the one-point posterior."""
    m = om.make_model(kind, 0.5, 1.0)
    t = np.arange(6) * 5e3
    y = np.array([0.3, -1.0, 2.0, 0.1, -0.4, 0.8])
    R = 0.05
    res = oracle.run(m, t, y, np.ones(6, np.uint8), R)
    v0 = m.Pinf[0, 0]
    ll = sum(-0.5 * (math.log(2 * math.pi * (v0 + R)) + yy * yy / (v0 + R)) for yy in y)
    assert abs(res.loglik - ll) < 1e-12
    np.testing.assert_allclose(res.f_mean, v0 * y / (v0 + R), rtol=1e-12)


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_all_missing_is_the_prior(oracle_lib, kind):
    """No observation: every filter/smoother state is N(0, P_inf) (stationarity,
    Sec. 4.1) and the log-likelihood is 0."""
    m = om.make_model(kind, 1.0, 1.0, balanced=True)
    t = np.sort(np.random.default_rng(3).uniform(0, 10, 50))
    res = oracle.run(m, t, np.zeros(50), np.zeros(50, np.uint8), 0.01)
    assert res.loglik == 0.0
    assert np.abs(res.m).max() == 0.0 and np.abs(res.ms).max() == 0.0
    for P in (res.P, res.Ps):
        assert np.abs(P - m.Pinf[None]).max() <= 1e-12 * np.abs(m.Pinf).max()


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_covariance_invariants(oracle_lib, kind):
    s = wl.prefix(wl.sinusoid_large(N=1 << 12, M=100), 600)
    m = om.make_model(kind, 1.0, 1.0, balanced=True)
    _, _, res, _ = oracle.predict(m, s.t_train, s.y_train, s.t_test, 0.01)
    for P in list(res.P) + list(res.Ps) + list(res.Q[1:]):
        np.testing.assert_array_equal(P, P.T)
        ev = np.linalg.eigvalsh(P)
        assert ev.min() >= -1e-12 * max(ev.max(), 1e-300)
    fvar_filter = res.P[:, 0, 0]
    assert np.all(res.f_var <= fvar_filter * (1 + 1e-12))
    assert np.all(fvar_filter <= m.Pinf[0, 0] * (1 + 1e-12))


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_balancing_invariance(oracle_lib, kind):
    """Sec. 4.2: the balanced model gives the same f-marginals and likelihood."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 12, M=100), 800)
    a = oracle.predict(om.make_model(kind, 1.0, 1.0), s.t_train, s.y_train, s.t_test, 0.01)
    b = oracle.predict(om.make_model(kind, 1.0, 1.0, balanced=True), s.t_train, s.y_train, s.t_test, 0.01)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-11)
    assert abs(a[2].loglik - b[2].loglik) <= 1e-12 * abs(a[2].loglik)


# --------------------------------------------------------------------------
# Props. 1 and 2: sequential and parallel filters/smoothers coincide.
# --------------------------------------------------------------------------

def _small_problem(kind, n, seed, missing=0.3):
    rng = np.random.default_rng(seed)
    m = om.make_model(kind, 0.9, 1.2, balanced=True)
    t = np.sort(rng.uniform(0, 0.4 * n, n))
    mask = (rng.uniform(size=n) > missing).astype(np.uint8)
    y = (np.sin(t) + rng.normal(0, 0.1, n)) * mask
    return m, t, y, mask


def _elements(m, t, y, mask, R):
    F, Q = oracle.discretize(m, t)
    A, b, C, eta, J = oracle.filter_elements(m, F, Q, y, mask, R)
    return F, Q, [(A[k], b[k], C[k], eta[k], J[k]) for k in range(t.size)]


def _tree_fold(op, elems, rng):
    """Combine a list with the associative operator in a random bracketing."""
    items = list(elems)
    while len(items) > 1:
        i = int(rng.integers(0, len(items) - 1))
        items[i:i + 2] = [op(items[i], items[i + 1])]
    return items[0]


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_prop1_filter_fold_equals_kalman_filter(oracle_lib, kind):
    m, t, y, mask = _small_problem(kind, 40, 11)
    F, Q, el = _elements(m, t, y, mask, 0.02)
    mo, Po, _, _, _ = oracle.kalman_filter(m, F, Q, y, mask, 0.02)
    acc = el[0]
    scale = np.abs(m.Pinf).max()
    for k in range(t.size):
        if k > 0:
            acc = oracle.filter_combine(acc, el[k])
        assert np.abs(acc[1] - mo[k]).max() <= 1e-12 * math.sqrt(scale)
        assert np.abs(acc[2] - Po[k]).max() <= 1e-12 * scale
        # every prefix holds A* = 0, eta* = 0, J* = 0 (it contains step 1)
        assert np.abs(acc[0]).max() == 0 and np.abs(acc[3]).max() == 0 and np.abs(acc[4]).max() == 0
    rng = np.random.default_rng(5)
    for _ in range(5):
        tot = _tree_fold(oracle.filter_combine, el, rng)
        assert np.abs(tot[1] - mo[-1]).max() <= 1e-12 * math.sqrt(scale)
        assert np.abs(tot[2] - Po[-1]).max() <= 1e-12 * scale


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_prop2_smoother_fold_equals_rts(oracle_lib, kind):
    m, t, y, mask = _small_problem(kind, 40, 12)
    F, Q, _ = _elements(m, t, y, mask, 0.02)
    mo, Po, mp, Pp, _ = oracle.kalman_filter(m, F, Q, y, mask, 0.02)
    ms, Ps = oracle.rts_smoother(F, mo, Po, mp, Pp)
    E, g, L = oracle.smoother_elements(F, Q, mo, Po)
    el = [(E[k], g[k], L[k]) for k in range(t.size)]
    scale = np.abs(m.Pinf).max()
    acc = el[-1]
    for k in range(t.size - 1, -1, -1):
        if k < t.size - 1:
            acc = oracle.smoother_combine(el[k], acc)
        assert np.abs(acc[1] - ms[k]).max() <= 1e-12 * math.sqrt(scale)
        assert np.abs(acc[2] - Ps[k]).max() <= 1e-12 * scale
    rng = np.random.default_rng(6)
    for _ in range(5):
        tot = _tree_fold(oracle.smoother_combine, el, rng)
        assert np.abs(tot[1] - ms[0]).max() <= 1e-12 * math.sqrt(scale)


def _all_bracketings(items, op):
    if len(items) == 1:
        return [items[0]]
    out = []
    for i in range(1, len(items)):
        for left in _all_bracketings(items[:i], op):
            for right in _all_bracketings(items[i:], op):
                out.append(op(left, right))
    return out


def test_all_bracketings_of_six_steps(oracle_lib):
    """Brute force: all 42 bracketings of 6 filter elements (from an interior
    segment, so that every component of the 5-tuple is non-trivial) agree."""
    m, t, y, mask = _small_problem("matern52", 12, 13, missing=0.2)
    _, _, el = _elements(m, t, y, mask, 0.02)
    seg = el[3:9]
    res = _all_bracketings(seg, oracle.filter_combine)
    assert len(res) == 42
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


def test_segment_reset(oracle_lib):
    """A first-step element (A = 0, eta = 0, J = 0) resets every prefix that
    contains it: scanning two concatenated series equals scanning each."""
    m, t, y, mask = _small_problem("matern32", 30, 14)
    F, Q, el = _elements(m, t, y, mask, 0.02)
    m2, t2, y2, mask2 = _small_problem("matern32", 20, 15)
    F2, Q2, el2 = _elements(m, t2, y2, mask2, 0.02)
    mo2, Po2, _, _, _ = oracle.kalman_filter(m, F2, Q2, y2, mask2, 0.02)
    acc = el[0]
    for e in el[1:] + el2:
        acc = oracle.filter_combine(acc, e)
    assert np.abs(acc[1] - mo2[-1]).max() <= 1e-12
    assert np.abs(acc[2] - Po2[-1]).max() <= 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_merge_brute_force(seed):
    rng = np.random.default_rng(seed)
    tt = np.sort(np.round(rng.uniform(0, 5, 40), 1))
    ts = np.sort(np.round(rng.uniform(0, 5, 17), 1))   # many ties
    y = rng.normal(size=40)
    t, ym, mask, tp = oracle.merge(tt, y, ts)
    # brute force: insert each test point after every training point <= it
    ref = [(x, 1, yy) for x, yy in zip(tt, y)]
    for j, x in enumerate(ts):
        pos = 0
        while pos < len(ref) and (ref[pos][0] < x or (ref[pos][0] == x and ref[pos][1] == 1) or
                                  (ref[pos][0] == x and ref[pos][1] == 0)):
            pos += 1
        ref.insert(pos, (x, 0, 0.0))
    np.testing.assert_array_equal(t, [r[0] for r in ref])
    np.testing.assert_array_equal(mask, [r[1] for r in ref])
    np.testing.assert_array_equal(ym, [r[2] for r in ref])
    np.testing.assert_array_equal(t[tp], ts)
    assert np.all(mask[tp] == 0) and np.all(np.diff(tp) > 0)


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_filter_from_a_start_state(oracle_lib, kind):
    """kalman_filter_from (the filter of a piece of a series given the state
    before it): with the start (0, anything) and the first transition
    F = 0, Q = P_inf it is kalman_filter; started from the filter state at
    step s-1 of a whole run, on steps s.. with their transitions, it gives the
    whole run's states there, and the two log-likelihoods add up to the whole
    (prediction-error decomposition, Sec. 2)."""
    s = wl.random_series(81, 3000, 300, T=40.0)
    t, y, mask, _ = oracle.merge(s.t_train, s.y_train, s.t_test)
    m = om.make_model(kind, 0.8, 1.3)
    F, Q = oracle.discretize(m, t)
    mo, Po, mp, Pp, ll = oracle.kalman_filter(m, F, Q, y, mask, 0.02)
    d = m.d
    rng = np.random.default_rng(82)
    Z = rng.normal(size=(d, d))
    mo2, Po2, _, _, ll2 = oracle.kalman_filter_from(m, np.zeros(d), Z @ Z.T + np.eye(d), F, Q, y, mask, 0.02)
    assert np.array_equal(mo2, mo) and np.array_equal(Po2, Po) and ll2 == ll
    for split in (1, 1234, 3299):
        a_m, a_P, _, _, a_ll = oracle.kalman_filter(m, F[:split], Q[:split], y[:split], mask[:split], 0.02)
        b_m, b_P, _, _, b_ll = oracle.kalman_filter_from(m, a_m[-1], a_P[-1], F[split:], Q[split:], y[split:],
                                                         mask[split:], 0.02)
        sd = np.sqrt(np.einsum("kii->ki", Po[split:]))
        assert np.max(np.abs(b_m - mo[split:]) / np.maximum(np.abs(mo[split:]), sd)) < 1e-12
        assert np.max(np.abs(b_P - Po[split:]) / (sd[:, :, None] * sd[:, None, :])) < 1e-12
        assert abs(a_ll + b_ll - ll) <= 1e-12 * max(abs(ll), 1.0)
