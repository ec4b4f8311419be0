"""Plain sequential CPU oracle for the parallel state-space GP path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything under ``oracle/``.  The oracle shares no code with the
CUDA library (``paper_2102_09964_b300``) and neither imports the other; the
product path never falls back to it.

Paper: Corenflos, Zhao, Sarkka, "Temporal Gaussian Process Regression in
Logarithmic Time".  What the oracle computes (all in long double inside
``ssgp_oracle.c``):

* discretisation, supplement Eq. (ss-gp-formation) (Van Loan block exponential);
* sequential Kalman filter with missing measurements, supplement Eqs. (nomeas)
  and (withmeas1), started from N(0, P_inf) (Sec. 4.1);
* log marginal likelihood by prediction-error decomposition (Sec. 2);
* sequential RTS smoother, supplement Eq. (smoother) with the sign of the
  covariance term taken from the proof of Prop. 2;
* the parallel-filter elements and operator (Sec. 3) and the parallel-smoother
  elements and operator (supplement, Prop. 2), for the Prop. 1/2 checks;
* the gradient of the log-likelihood in (log lengthscale, log variance,
  log noise) by forward mode: the Frechet derivative of the Van Loan
  exponential and the differentiated sequential filter
  (``loglik_grad_fwd``), plus central differences (``loglik_grad_fd``).

Model formation (``model.py``), merge (``merge.py``) and the dense GP
(``dense_gp.py``) are numpy.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (dense GP, closed forms, invariants, Prop. 1/2 folds,
brute-force bracketings); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import model as model  # noqa: F401  (re-export)
from .merge import merge  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssgp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile ssgp_oracle.c into oracle/liboracle.so with gcc (OpenMP for the
    embarrassingly parallel discretisation loop)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", out, src, "-lm"]
        subprocess.check_call(cmd)
    return out


def use_library(path: str | None):
    """Point the wrappers at another build of ssgp_oracle.c (used by the test
    that plants mistakes in the oracle to show the pins catch them)."""
    global _lib
    _lib = None if path is None else ctypes.CDLL(path)


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        assert _lib.orc_version() == 1
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def discretize(m, t: np.ndarray):
    """F[k], Q[k] (d x d) of the transition into step k; F[0] = 0, Q[0] = P_inf."""
    lib = _load()
    d = m.d
    t = _c(t)
    n = t.size
    F = np.empty((n, d, d)); Q = np.empty((n, d, d))
    rc = lib.orc_discretize(d, _p(_c(m.G)), _p(_c(m.W)), _p(_c(m.Pinf)), _p(t),
                            ctypes.c_long(n), _p(F), _p(Q))
    _check(rc, "discretize")
    return F, Q


def _R_arr(R, n):
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    per = 1 if (R.size == n and n > 1) else 0
    if R.size != 1 and not per:
        raise ValueError("R must be scalar or per step")
    return _c(R), per


def kalman_filter(m, F, Q, y, mask, R):
    """Sequential KF; returns (m, P, m_pred, P_pred, loglik)."""
    lib = _load()
    d = m.d
    n = F.shape[0]
    Ra, per = _R_arr(R, n)
    y = _c(y); mask = np.ascontiguousarray(mask, dtype=np.uint8)
    mo = np.empty((n, d)); Po = np.empty((n, d, d)); mp = np.empty((n, d)); Pp = np.empty((n, d, d))
    ll = ctypes.c_double(0.0)
    rc = lib.orc_kalman_filter(d, _p(_c(m.H).ravel()), _p(Ra), per, _p(_c(m.Pinf)), _p(_c(F)), _p(_c(Q)),
                               _p(y), _u8(mask), ctypes.c_long(n), _p(mo), _p(Po), _p(mp), _p(Pp),
                               ctypes.byref(ll))
    _check(rc, "kalman_filter")
    return mo, Po, mp, Pp, ll.value


def kalman_filter_from(m, x0, P0, F, Q, y, mask, R):
    """Sequential KF of a piece of a series started from the state
    N(x0, P0) before its step 0 (every step, step 0 included, a transition
    F[k], Q[k]); returns (m, P, m_pred, P_pred, loglik)."""
    lib = _load()
    d = m.d
    n = F.shape[0]
    Ra, per = _R_arr(R, n)
    y = _c(y); mask = np.ascontiguousarray(mask, dtype=np.uint8)
    mo = np.empty((n, d)); Po = np.empty((n, d, d)); mp = np.empty((n, d)); Pp = np.empty((n, d, d))
    ll = ctypes.c_double(0.0)
    rc = lib.orc_kalman_filter_from(d, _p(_c(m.H).ravel()), _p(Ra), per, _p(_c(x0)), _p(_c(P0)), _p(_c(F)),
                                    _p(_c(Q)), _p(y), _u8(mask), ctypes.c_long(n), _p(mo), _p(Po), _p(mp),
                                    _p(Pp), ctypes.byref(ll))
    _check(rc, "kalman_filter_from")
    return mo, Po, mp, Pp, ll.value


def rts_smoother(F, mo, Po, mp, Pp):
    lib = _load()
    n, d = mo.shape
    ms = np.empty((n, d)); Ps = np.empty((n, d, d))
    rc = lib.orc_rts_smoother(d, _p(_c(F)), _p(_c(mo)), _p(_c(Po)), _p(_c(mp)), _p(_c(Pp)),
                              ctypes.c_long(n), _p(ms), _p(Ps))
    _check(rc, "rts_smoother")
    return ms, Ps


def filter_elements(m, F, Q, y, mask, R):
    """Per-step (A, b, C, eta, J) of Sec. 3 / supplement Prop. 1."""
    lib = _load()
    d = m.d
    n = F.shape[0]
    Ra, per = _R_arr(R, n)
    A = np.empty((n, d, d)); b = np.empty((n, d)); C = np.empty((n, d, d))
    eta = np.empty((n, d)); J = np.empty((n, d, d))
    rc = lib.orc_filter_elements(d, _p(_c(m.H).ravel()), _p(Ra), per, _p(_c(m.Pinf)), _p(_c(F)), _p(_c(Q)),
                                 _p(_c(y)), _u8(np.ascontiguousarray(mask, dtype=np.uint8)),
                                 ctypes.c_long(n), _p(A), _p(b), _p(C), _p(eta), _p(J))
    _check(rc, "filter_elements")
    return A, b, C, eta, J


def filter_combine(ei, ej):
    """The filtering operator of Sec. 3 on two 5-tuples (i earlier, j later)."""
    lib = _load()
    d = ei[0].shape[0]
    out = [np.empty((d, d)), np.empty(d), np.empty((d, d)), np.empty(d), np.empty((d, d))]
    ins = [_c(x) for x in ei] + [_c(x) for x in ej]
    args = [_p(x) for x in ins] + [_p(x) for x in out]
    _check(lib.orc_filter_combine(d, *args), "filter_combine")
    return tuple(out)


def smoother_elements(F, Q, mo, Po):
    lib = _load()
    n, d = mo.shape
    E = np.empty((n, d, d)); g = np.empty((n, d)); L = np.empty((n, d, d))
    rc = lib.orc_smoother_elements(d, _p(_c(F)), _p(_c(Q)), _p(_c(mo)), _p(_c(Po)), ctypes.c_long(n),
                                   _p(E), _p(g), _p(L))
    _check(rc, "smoother_elements")
    return E, g, L


def smoother_combine(ei, ej):
    """The smoothing operator of the supplement (i earlier, j later)."""
    lib = _load()
    d = ei[0].shape[0]
    out = [np.empty((d, d)), np.empty(d), np.empty((d, d))]
    ins = [_c(x) for x in ei] + [_c(x) for x in ej]
    args = [_p(x) for x in ins] + [_p(x) for x in out]
    _check(lib.orc_smoother_combine(d, *args), "smoother_combine")
    return tuple(out)


@dataclass
class Result:
    m: np.ndarray       # filter means   (n, d)
    P: np.ndarray       # filter covs    (n, d, d)
    ms: np.ndarray      # smoother means (n, d)
    Ps: np.ndarray      # smoother covs  (n, d, d)
    loglik: float
    f_mean: np.ndarray  # H m^s
    f_var: np.ndarray   # H P^s H^T
    F: np.ndarray
    Q: np.ndarray


def run(m, t, y, mask, R) -> Result:
    """Discretise, filter, smooth: the whole sequential state-space GP."""
    F, Q = discretize(m, t)
    mo, Po, mp, Pp, ll = kalman_filter(m, F, Q, y, mask, R)
    ms, Ps = rts_smoother(F, mo, Po, mp, Pp)
    H = m.H.ravel()
    f_mean = ms @ H
    f_var = np.einsum("i,kij,j->k", H, Ps, H)
    return Result(m=mo, P=Po, ms=ms, Ps=Ps, loglik=ll, f_mean=f_mean, f_var=f_var, F=F, Q=Q)


def predict(m, t_train, y_train, t_test, R):
    """Merge (Sec. 4.3), run, and gather the test-point marginals."""
    t, y, mask, test_pos = merge(t_train, y_train, t_test)
    res = run(m, t, y, mask, R)
    return res.f_mean[test_pos], res.f_var[test_pos], res, (t, y, mask, test_pos)


# ---------------------------------------------------------------------------
# Gradient of the log marginal likelihood with respect to
# theta = (log lengthscale, log variance, log noise variance)
# ---------------------------------------------------------------------------
GRAD_PARAMS = ("log_lengthscale", "log_variance", "log_noise")


def loglik_tangent(m, t, y, mask, R, param, with_scale=False):
    """(loglik, d loglik / d param) by forward mode through the discretisation
    (Frechet derivative of the Van Loan exponential) and the sequential
    Kalman filter, with the model's tangent from ``model.model_tangent``.
    ``m`` must be the unbalanced model; R scalar or per step.  With
    ``with_scale`` also the sum of |per-step term| of the derivative."""
    from . import model as _model
    lib = _load()
    d = m.d
    t = _c(t)
    n = t.size
    Ra, per = _R_arr(R, n)
    if param == "log_noise":
        dG = np.zeros((d, d)); dW = np.zeros((d, d)); dPinf = np.zeros((d, d))
        dRa = Ra.copy()
    else:
        dG, dW, dPinf = _model.model_tangent(m, param)
        dRa = np.zeros_like(Ra)
    F = np.empty((n, d, d)); Q = np.empty((n, d, d)); dF = np.empty((n, d, d)); dQ = np.empty((n, d, d))
    rc = lib.orc_discretize_tangent(d, _p(_c(m.G)), _p(_c(m.W)), _p(_c(m.Pinf)), _p(_c(dG)), _p(_c(dW)),
                                    _p(_c(dPinf)), _p(t), ctypes.c_long(n), _p(F), _p(Q), _p(dF), _p(dQ))
    _check(rc, "discretize_tangent")
    y = _c(y)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ll = ctypes.c_double(0.0)
    dll = ctypes.c_double(0.0)
    dabs = ctypes.c_double(0.0)
    rc = lib.orc_loglik_tangent(d, _p(_c(m.H).ravel()), _p(Ra), _p(dRa), per, _p(F), _p(Q), _p(dF), _p(dQ),
                                _p(y), _u8(mask), ctypes.c_long(n), ctypes.byref(ll), ctypes.byref(dll),
                                ctypes.byref(dabs))
    _check(rc, "loglik_tangent")
    if with_scale:
        return ll.value, dll.value, dabs.value
    return ll.value, dll.value


def loglik_grad_fwd(kind, lengthscale, variance, t, y, mask, R, order=6, with_scale=False):
    """(loglik, gradient over GRAD_PARAMS) by forward mode, one direction at a
    time (R scalar or per step; d/d log noise scales every R_k).  With
    ``with_scale`` also, per component, the sum over steps of the absolute
    per-step terms (``loglik_tangent``)."""
    from . import model as _model
    m = _model.make_model(kind, lengthscale, variance, order=order)
    g = []
    sc = []
    ll = None
    for p in GRAD_PARAMS:
        ll, dl, ds = loglik_tangent(m, t, y, mask, R, p, with_scale=True)
        g.append(dl)
        sc.append(ds)
    if with_scale:
        return ll, np.array(g), np.array(sc)
    return ll, np.array(g)


def loglik_at(kind, lengthscale, variance, t, y, mask, R, order=6):
    """The oracle log-likelihood of the model built at these hyperparameters."""
    from . import model as _model
    m = _model.make_model(kind, lengthscale, variance, order=order)
    F, Q = discretize(m, t)
    return kalman_filter(m, F, Q, y, mask, R)[4]


def loglik_grad_fd(kind, lengthscale, variance, t, y, mask, R, h=1e-6, order=6, threads=1):
    """Central finite differences of the oracle log-likelihood in
    (log lengthscale, log variance, log noise), step h in each log parameter
    (the six evaluations in ``threads`` threads)."""
    base = np.log([lengthscale, variance])
    R = np.asarray(R, dtype=np.float64)
    points = []
    for i in range(3):
        for sgn in (1.0, -1.0):
            th = base.copy()
            Rp = R
            if i < 2:
                th[i] += sgn * h
            else:
                Rp = R * math.exp(sgn * h)
            points.append((math.exp(th[0]), math.exp(th[1]), Rp))
    run = lambda p: loglik_at(kind, p[0], p[1], t, y, mask, p[2], order=order)
    if threads > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            vals = list(ex.map(run, points))
    else:
        vals = [run(p) for p in points]
    return np.array([(vals[2 * i] - vals[2 * i + 1]) / (2.0 * h) for i in range(3)])


# ---------------------------------------------------------------------------
# Simulation from the state-space prior (training data of the learned
# initialisation), with the Philox4x32-10 counter-based generator
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter and 2-word key (list of 4 ints)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed: int, sid: int, k: int, count: int) -> np.ndarray:
    """The `count` standard normals of series `sid` at step k."""
    lib = _load()
    z = np.empty(count + 1)
    lib.orc_normals(ctypes.c_uint64(seed), ctypes.c_uint32(sid), ctypes.c_uint32(k), count, _p(z))
    return z[:count]


def simulate_series(m, R: float, n: int, seed: int, sid: int, spacing: float = 0.01):
    """(t, y) of series `sid` drawn from the prior of model m (its own
    coordinates) with noise variance R, n steps of a Poisson time grid."""
    lib = _load()
    t = np.empty(n)
    y = np.empty(n)
    rc = lib.orc_simulate_series(m.d, _p(_c(m.G)), _p(_c(m.W)), _p(_c(m.Pinf)), _p(_c(m.H).ravel()),
                                 ctypes.c_double(R), ctypes.c_long(n), ctypes.c_uint64(seed), ctypes.c_uint32(sid),
                                 ctypes.c_double(spacing), _p(t), _p(y))
    _check(rc, "simulate_series")
    return t, y
