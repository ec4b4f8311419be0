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
  elements and operator (supplement, Prop. 2), for the Prop. 1/2 checks.

Model formation (``model.py``), merge (``merge.py``) and the dense GP
(``dense_gp.py``) are numpy.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (dense GP, closed forms, invariants, Prop. 1/2 folds,
brute-force bracketings); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
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
