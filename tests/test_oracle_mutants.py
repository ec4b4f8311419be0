"""The pins are sensitive: plausible mistakes planted in a copy of the oracle
(a dropped term, a wrong sign, a wrong index, a transposed operand) make at
least one pin fail, while the unmodified source passes them all.

Mistakes are planted only in a temporary copy of ``oracle/ssgp_oracle.c`` on
the CPU; the oracle itself is never modified.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense_gp
from oracle import model as om

SRC = os.path.join(os.path.dirname(oracle.__file__), "ssgp_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("rts_sign", "for (int i = 0; i < dd; ++i) nPs[i] += P[i];",
     "for (int i = 0; i < dd; ++i) nPs[i] = P[i] - nPs[i];"),
    ("drop_Q_predict", "      for (int i = 0; i < dd; ++i) Pp[i] += Q[i];\n      symmetrize(d, Pp);\n    }",
     "      for (int i = 0; i < dd; ++i) Pp[i] += 0.0L * Q[i];\n      symmetrize(d, Pp);\n    }"),
    ("untransposed_F_predict", "      tr(d, d, F, Ft);\n      mm(d, d, d, FP, Ft, Pp);                     /* P^- = F P F^T + Q  */",
     "      tr(d, d, F, Ft);\n      mm(d, d, d, FP, F, Pp);                     /* P^- = F P F^T + Q  */"),
    ("loglik_no_2pi", "logl(twopi * S)", "logl(S)"),
    ("vanloan_F_not_transposed", "F[i * d + j] = E[(d + j) * n + d + i];", "F[i * d + j] = E[(d + i) * n + d + j];"),
    ("innovation_sign", "v -= H[i] * mp[i];", "v += H[i] * mp[i];"),
    ("doubling_drops_Q", "for (int i = 0; i < d * d; ++i) Q[i] += FQF[i];", "for (int i = 0; i < d * d; ++i) Q[i] = FQF[i];"),
    ("combine_JC_order", "mm(d, d, d, Ci, Jj, M1);", "mm(d, d, d, Jj, Ci, M1);"),
    ("combine_eta_sign", "RHS2[i * m2] = etaj[i] - Jb[i];", "RHS2[i * m2] = etaj[i] + Jb[i];"),
    ("element_J_no_S", "J[i * d + j] = HF[i] * HF[j] / S;", "J[i * d + j] = HF[i] * HF[j];"),
    ("element_C_no_update", "mm(d, d, d, IKH, Q, C);", "memcpy(C, Q, sizeof(real) * dd);"),
    ("smoother_g_sign", "g[i] = m[i] - EFm[i];", "g[i] = m[i] + EFm[i];"),
    ("vanloan_Q_order", "mm(d, d, d, F, E12, Q);", "mm(d, d, d, E12, F, Q);"),
    ("smoother_combine_transposed", "mm(d, d, d, Ei, Lj, T);\n  tr(d, d, Ei, Eit);\n  mm(d, d, d, T, Eit, L);",
     "tr(d, d, Ei, Eit);\n  mm(d, d, d, Eit, Lj, T);\n  mm(d, d, d, T, Ei, L);"),
    ("filter_from_ignores_start_mean", "load(1, d, x0_, m);", "for (int i = 0; i < d; ++i) m[i] = 0.0L;"),
    ("filter_from_drops_start_cov", "mm(d, d, d, FP, Ft, Pp);                       /* P^- = F P F^T + Q  */",
     "mm(d, d, d, FP, Ft, Pp);                       /* P^- = F P F^T + Q  */\n    if (k == 0) memset(Pp, 0, sizeof(Pp));"),
]


def _battery():
    """The pins in miniature: dense GP (Lemma), stationarity, the Lyapunov
    identity of Q, Props. 1 and 2."""
    rng = np.random.default_rng(21)
    n = 120
    t = np.sort(rng.uniform(0, 12, n))
    mask = (rng.uniform(size=n) > 0.25).astype(np.uint8)
    y = (np.sin(2 * t) + rng.normal(0, 0.1, n)) * mask
    for kind, nu in [("matern32", 1.5), ("matern52", 2.5)]:
        m = om.make_model(kind, 0.7, 1.3)
        res = oracle.run(m, t, y, mask, 0.02)
        mean, var, ll = dense_gp.posterior(om.matern_kernel(nu, 0.7, 1.3), t, mask, y, 0.02)
        assert np.max(np.abs(res.f_mean - mean) / np.maximum(np.abs(mean), np.sqrt(var))) < 1e-9
        assert np.max(np.abs(res.f_var - var) / var) < 1e-9
        assert abs(res.loglik - ll) < 1e-9 * max(abs(ll), n)
        for k in (1, 50, 100):
            assert np.abs(res.F[k] @ m.Pinf @ res.F[k].T + res.Q[k] - m.Pinf).max() < 1e-12 * np.abs(m.Pinf).max()
            # the Lyapunov identity of the integral, G Q + Q G^T = F W F^T - W
            lhs = m.G @ res.Q[k] + res.Q[k] @ m.G.T
            rhs = res.F[k] @ m.W @ res.F[k].T - m.W
            assert np.abs(lhs - rhs).max() < 1e-12 * (np.abs(m.G).max() * np.abs(res.Q[k]).max() + np.abs(m.W).max())
        tl = np.array([0.0, 40.0])        # a long step exercises the doubling
        F, Q = oracle.discretize(m, tl)
        assert np.abs(F[1] @ m.Pinf @ F[1].T + Q[1] - m.Pinf).max() < 1e-12 * np.abs(m.Pinf).max()
        # Prop. 1 (filter fold) and Prop. 2 (smoother fold) on the first 25 steps
        k0 = 25
        A, b, C, eta, J = oracle.filter_elements(m, res.F[:k0], res.Q[:k0], y[:k0], mask[:k0], 0.02)
        acc = (A[0], b[0], C[0], eta[0], J[0])
        for k in range(1, k0):
            acc = oracle.filter_combine(acc, (A[k], b[k], C[k], eta[k], J[k]))
        assert np.abs(acc[1] - res.m[k0 - 1]).max() < 1e-11 and np.abs(acc[2] - res.P[k0 - 1]).max() < 1e-11
        # an interior bracketing must agree with the left fold of the same segment
        seg = [(A[k], b[k], C[k], eta[k], J[k]) for k in range(5, 9)]
        l = oracle.filter_combine(oracle.filter_combine(oracle.filter_combine(seg[0], seg[1]), seg[2]), seg[3])
        r = oracle.filter_combine(seg[0], oracle.filter_combine(seg[1], oracle.filter_combine(seg[2], seg[3])))
        for u, v in zip(l, r):
            assert np.abs(u - v).max() < 1e-11 * max(1.0, np.abs(v).max())
        # the filter of the steps after a split, from the filter state there
        _, _, _, _, lla = oracle.kalman_filter(m, res.F[:60], res.Q[:60], y[:60], mask[:60], 0.02)
        mo2, Po2, _, _, llb = oracle.kalman_filter_from(m, res.m[59], res.P[59], res.F[60:], res.Q[60:], y[60:],
                                                        mask[60:], 0.02)
        assert np.abs(mo2 - res.m[60:]).max() < 1e-11 and np.abs(Po2 - res.P[60:]).max() < 1e-11
        assert abs(lla + llb - res.loglik) < 1e-11 * max(1.0, abs(res.loglik))
        E, g, L = oracle.smoother_elements(res.F, res.Q, res.m, res.P)
        acc = (E[-1], g[-1], L[-1])
        for k in range(n - 2, n - 30, -1):
            acc = oracle.smoother_combine((E[k], g[k], L[k]), acc)
        assert np.abs(acc[1] - res.ms[n - 29]).max() < 1e-11 and np.abs(acc[2] - res.Ps[n - 29]).max() < 1e-11
        seg = [(E[k], g[k], L[k]) for k in range(10, 14)]
        l = oracle.smoother_combine(oracle.smoother_combine(seg[0], seg[1]), oracle.smoother_combine(seg[2], seg[3]))
        r = oracle.smoother_combine(seg[0], oracle.smoother_combine(seg[1], oracle.smoother_combine(seg[2], seg[3])))
        for u, v in zip(l, r):
            assert np.abs(u - v).max() < 1e-11 * max(1.0, np.abs(v).max())


def _with_source(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / f"{name}.so"))
    oracle.use_library(lib)


def test_unmodified_oracle_passes_battery(tmp_path):
    try:
        _with_source(tmp_path, "control", open(SRC).read())
        _battery()
    finally:
        oracle.use_library(None)


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, bad):
    text = open(SRC).read()
    assert text.count(orig) >= 1, f"mutation site for {name} not found"
    mutated = text.replace(orig, bad, 1)
    try:
        _with_source(tmp_path, name, mutated)
        with pytest.raises((AssertionError, RuntimeError, np.linalg.LinAlgError, ValueError)):
            _battery()
    finally:
        oracle.use_library(None)
