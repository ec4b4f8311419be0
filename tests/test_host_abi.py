"""CPU tests of libpssgp's host side: the library loads and exports every
symbol declared in include/pssgp.h; model formation (Sec. 2, 4.1, 4.2) agrees
with the oracle's independent construction; the Taylor tables of the device
discretisation reproduce the matrix exponential and the Q integral; host-side
argument errors are rejected before any launch.  No GPU needed."""
import math
import os
import re

import numpy as np
import pytest
from scipy.linalg import expm

import paper_2102_09964_b300 as P
from oracle import model as om

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2102_09964_b300 import build
    build.build()
    return P.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "pssgp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int32_t|int|size_t|const char\s*\*)\s*(pssgp_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm


def sde_coords(m):
    """Balanced model -> SDE coordinates x = D z."""
    D = np.array(m.D)
    G = m.matrix("G") * D[:, None] / D[None, :]
    Pinf = m.matrix("Pinf") * D[:, None] * D[None, :]
    W = m.matrix("W") * D[:, None] * D[None, :]
    return G, Pinf, W


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
@pytest.mark.parametrize("ell,s2", [(0.5, 1.0), (1.0, 2.0), (4.0, 0.7)])
@pytest.mark.parametrize("balance", [False, True])
def test_model_matches_oracle(lib, kind, ell, s2, balance):
    m = P.build_model(kind, ell, s2, order=6, balance=balance)
    o = om.make_model(kind, ell, s2)
    G, Pinf, W = sde_coords(m)
    sc = np.abs(o.G).max()
    assert np.abs(G - o.G).max() <= 1e-12 * sc
    assert np.abs(Pinf - o.Pinf).max() <= 1e-11 * np.abs(o.Pinf).max()
    assert np.abs(W - o.W).max() <= 1e-11 * np.abs(o.W).max()
    D = np.array(m.D)
    assert D[0] == 1.0
    assert np.all(np.log2(D) == np.round(np.log2(D)))


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("h", [0.0, 1e-4, 3e-3, 0.008, 0.03])
def test_taylor_tables_reproduce_discretisation(lib, kind, h):
    """F(h) (row 0 by the series, other rows by the companion recursion) and
    Q(h) = h sum_m qc h^m, with the term counts picked from the model's step
    thresholds, equal exp(G h) and the Van Loan integral of Eq.
    (ss-gp-formation), computed here by scipy."""
    m = P.build_model(kind, 1.0, 1.0)
    d = m.d
    G, W = m.matrix("G"), m.matrix("W")
    assert h <= m.raw.hmax
    kf = next(k for k in range(1, 17) if h <= m.raw.hthr_f[k])
    kq = next(k for k in range(1, 17) if h <= m.raw.hthr_q[k])
    fc = np.array(m.raw.fc[:]).reshape(8 * 8, 16)[: d * d]
    qc = np.array(m.raw.qc[:]).reshape(8 * 8, 16)[: d * d]
    assert m.raw.companion == 1
    rsup = np.array(m.raw.rsup[:64])[: d * d].reshape(d, d)
    rlast = np.array(m.raw.rlast[:64])[: d * d].reshape(d, d)
    F = np.zeros((d, d))
    F[0] = sum(fc[:d, t] * h ** t for t in range(kf))
    for i in range(d - 1):
        F[i + 1, 0] = F[i, d - 1] * rlast[i, 0]
        for j in range(1, d):
            F[i + 1, j] = F[i, j - 1] * rsup[i, j] + F[i, d - 1] * rlast[i, j]
    Ffull = sum(fc[:, t] * h ** t for t in range(kf)).reshape(d, d)
    Q = h * sum(qc[:, t] * h ** t for t in range(kq)).reshape(d, d)
    Fr = expm(G * h)
    C = np.zeros((2 * d, 2 * d))
    C[:d, :d] = -G * h
    C[:d, d:] = W * h
    C[d:, d:] = G.T * h
    E = expm(C)
    Qr = E[d:, d:].T @ E[:d, d:]
    assert np.abs(F - Fr).max() <= 4e-16 * max(1.0, np.abs(Fr).max())
    assert np.abs(Ffull - Fr).max() <= 4e-16 * max(1.0, np.abs(Fr).max())
    assert np.abs(Q - Qr).max() <= 1e-14 * max(np.abs(Qr).max(), 1e-300) + 1e-300


def test_thresholds_are_monotone_and_bounded(lib):
    m = P.build_model("rbf", 1.0, 1.0)
    assert m.raw.hmax > 0.03
    assert all(m.raw.hthr_f[k] <= m.raw.hthr_f[k + 1] for k in range(16))
    assert all(m.raw.hthr_q[k] <= m.raw.hthr_q[k + 1] for k in range(16))
    # a user drift that is not in companion form uses the full series
    o = om.make_model("matern52", 1.0, 1.0)
    Gm = o.G.copy()
    Gm[0, 2] = 0.1
    assert P.model_from_sde(Gm, o.L, o.q, o.H).raw.companion == 0


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7, 8])
def test_rbf_spectral_factor_all_orders(lib, order):
    """The product's own root finder (Aberth on the truncated exponential) gives
    the same Hurwitz factor as the oracle's numpy.roots on the degree-2n
    polynomial."""
    m = P.build_model("rbf", 0.8, 1.3, order=order, balance=False)
    o = om.make_model("rbf", 0.8, 1.3, order=order)
    G, Pinf, _ = sde_coords(m)
    assert np.abs(G - o.G).max() <= 1e-11 * np.abs(o.G).max()
    assert np.abs(Pinf - o.Pinf).max() <= 1e-10 * np.abs(o.Pinf).max()


def test_model_from_sde_matches_build(lib):
    o = om.make_model("matern52", 0.9, 1.4)
    a = P.model_from_sde(o.G, o.L, o.q, o.H, balance=True)
    b = P.build_model("matern52", 0.9, 1.4, balance=True)
    np.testing.assert_allclose(a.matrix("G"), b.matrix("G"), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(a.matrix("Pinf"), b.matrix("Pinf"), rtol=1e-12, atol=1e-14)
    # H = 2 e_0 is absorbed into D (f = x_0 / ... stays the output)
    c = P.model_from_sde(o.G, o.L, o.q, 2.0 * o.H, balance=False)
    assert c.D[0] == 0.5


def test_host_argument_errors(lib):
    import ctypes
    k = P.PssgpKernel(P.MATERN32, 0, -1.0, 1.0, 1, 0)
    m = P.PssgpModel()
    assert lib.pssgp_model_build(ctypes.byref(k), ctypes.byref(m)) == -3       # EKERNEL
    k = P.PssgpKernel(P.RBF, 9, 1.0, 1.0, 1, 0)
    assert lib.pssgp_model_build(ctypes.byref(k), ctypes.byref(m)) == -2       # EDIM
    k = P.PssgpKernel(77, 0, 1.0, 1.0, 1, 0)
    assert lib.pssgp_model_build(ctypes.byref(k), ctypes.byref(m)) == -3
    assert lib.pssgp_workspace_size(9, 10) == 0
    assert lib.pssgp_workspace_size(3, 0) == 0
    mm = P.build_model("matern32", 1.0, 1.0)
    # null pointers / bad sizes are rejected on the host (no launch)
    assert lib.pssgp_filter(ctypes.byref(mm.raw), None, None, None, None, 0, 10, None, None, 10, None,
                            None, 0, None) == -1
    assert lib.pssgp_predict(ctypes.byref(mm.raw), None, None, 0, None, 0, 0.01, None, None, None,
                             None, 0, None) == -1
    assert lib.pssgp_loglik_batched(ctypes.byref(mm.raw), None, 1, None, None, None, None, 10, None,
                                    None, 0, None) == -1
    # a model without a lengthscale / variance cannot be rescaled per series
    # (checked before anything is dereferenced: the pointers here are dummies)
    o = om.make_model("matern32", 1.0, 1.0)
    sde = P.model_from_sde(o.G, o.L, o.q, o.H)
    fake = ctypes.c_void_p(256)
    assert lib.pssgp_loglik_batched(ctypes.byref(sde.raw), fake, 1, fake, fake, fake, fake, 10, fake,
                                    fake, 1 << 30, None) == -6
    assert lib.pssgp_loglik_batched(ctypes.byref(mm.raw), fake, 0, fake, fake, fake, fake, 10, fake,
                                    fake, 1 << 30, None) == -1


def test_workspace_size_grows_linearly(lib):
    a = P.workspace_size(6, 1 << 16)
    b = P.workspace_size(6, 1 << 17)
    assert 1.8 < b / a < 2.2


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_fp32_split_thresholds_bound_the_tail(kind):
    """At h = hthr_f32[K] the terms of exp(hG) from K on sum below 2^-36 in
    the 1-norm (recomputed here from the model's own balanced drift), the
    thresholds grow with K and are looser than the FP64 truncation ones."""
    m = P.build_model(kind, 1.0, 1.0)
    d = m.d
    G = m.matrix("G")
    hf32 = np.array(m.raw.hthr_f32[:17])
    hf = np.array(m.raw.hthr_f[:17])
    assert np.all(np.diff(hf32[1:]) > 0) and np.all(hf32[1:] >= hf[1:])
    for K in (3, 6, 9, 12):
        h = hf32[K]
        tail, Gm, fact = 0.0, np.linalg.matrix_power(G, K), math.factorial(K)
        for mm in range(K, 80):
            tail += np.abs(Gm).sum(axis=0).max() * h ** mm / fact
            Gm = Gm @ G
            fact *= mm + 1
        assert tail <= 2.0 ** -36 * 1.01, (K, tail)


def test_host_argument_errors_of_the_newer_entry_points(lib):
    """Rejected on the host before anything is launched (dummy pointers are
    never dereferenced)."""
    import ctypes
    fake = ctypes.c_void_p(256)
    mm = P.build_model("matern52", 1.0, 1.0)
    EINVAL, EMODEL, EWS = -1, -6, -4
    # gradient: null grad output, bad n
    assert lib.pssgp_loglik_grad(ctypes.byref(mm.raw), fake, fake, fake, fake, 0, 10, None, None, fake, 1 << 30,
                                 None) == EINVAL
    assert lib.pssgp_loglik_grad_batched(ctypes.byref(mm.raw), fake, 0, fake, fake, fake, fake, 10, None, fake,
                                         fake, 1 << 30, None) == EINVAL
    # fit: options out of range, offsets that do not end at n
    offs = np.array([0, 5, 10], dtype=np.int64)
    bad = [dict(max_iter=0), dict(patience=0), dict(lr=0.0), dict(check_every=0), dict(method=7)]
    for kw in bad:
        o = P.FitOptions(kw.get("max_iter", 10), kw.get("patience", 2), 1e-7, kw.get("lr", 0.05), 0.9, 0.999, 1e-8,
                         kw.get("check_every", 5), kw.get("method", 0))
        assert lib.pssgp_fit_batched(ctypes.byref(mm.raw), offs.ctypes.data_as(ctypes.c_void_p), 2, fake, fake,
                                     fake, 10, fake, fake, fake, ctypes.byref(o), fake, 1 << 30, None,
                                     None) == EINVAL
    o = P.FitOptions(10, 2, 1e-7, 0.05, 0.9, 0.999, 1e-8, 5, 1)
    assert lib.pssgp_fit_batched(ctypes.byref(mm.raw), offs.ctypes.data_as(ctypes.c_void_p), 2, fake, fake, fake,
                                 11, fake, fake, fake, ctypes.byref(o), fake, 1 << 30, None, None) == EINVAL
    assert lib.pssgp_fit_batched(ctypes.byref(mm.raw), offs.ctypes.data_as(ctypes.c_void_p), 2, fake, fake, fake,
                                 10, fake, fake, fake, ctypes.byref(o), fake, 16, None, None) == EWS
    # simulation: the model must carry its hyperparameters; spacing > 0
    o5 = om.make_model("matern52", 1.0, 1.0)
    sde = P.model_from_sde(o5.G, o5.L, o5.q, o5.H)
    assert lib.pssgp_simulate_prior(ctypes.byref(sde.raw), fake, 1, fake, 1, 0.01, fake, fake, fake,
                                    None) == EMODEL
    assert lib.pssgp_simulate_prior(ctypes.byref(mm.raw), fake, 1, fake, 1, 0.0, fake, fake, fake, None) == EINVAL
    assert lib.pssgp_features(None, 1, fake, fake, fake, None) == EINVAL
    # network: minibatch rows a multiple of 8, workspace size and alignment
    assert lib.pssgp_mlp_grad(fake, fake, fake, 12, fake, None, None, fake, 1 << 30, None) == EINVAL
    assert lib.pssgp_mlp_grad(fake, fake, fake, 16, fake, None, None, fake, 16, None) == EWS
    assert lib.pssgp_mlp_predict(fake, fake, 16, fake, ctypes.c_void_p(257), 1 << 30, None) == EWS
    assert lib.pssgp_mlp_adam(fake, fake, 1e-3, 0, None) == EINVAL
    assert lib.pssgp_mlp_workspace_size(0) == 0 and lib.pssgp_mlp_state_bytes() > 0
    assert lib.pssgp_mlp_param_count() == 256 * 80 + 256 + 256 * 256 + 256 + 16 * 256 + 16
    # host-buffer prediction: workspace too small
    assert lib.pssgp_predict_host(ctypes.byref(mm.raw), fake, fake, 10, fake, 5, 0.01, fake, fake, None, fake,
                                  1024, None) == EWS
    assert lib.pssgp_predict_host_workspace_size(3, 10, 5) >= lib.pssgp_workspace_size(3, 15)
    # workspaces
    assert lib.pssgp_workspace_size_grad(3, 1000) > lib.pssgp_workspace_size(3, 1000)
    assert lib.pssgp_fit_workspace_size(3, 1000, 4) > lib.pssgp_workspace_size_grad(3, 1000)
    assert lib.pssgp_tune_set(0, 8) == -2 and lib.pssgp_tune_get(9) == -2
    assert lib.pssgp_tune_set(3, 0) == EINVAL and lib.pssgp_tune_set(3, 17) == EINVAL
    assert lib.pssgp_set_warps_per_sm(0) == EINVAL and lib.pssgp_set_warps_per_sm(17) == EINVAL
    old = lib.pssgp_tune_get(3)
    assert lib.pssgp_tune_set(3, 2) == 0 and lib.pssgp_tune_get(3) == 2
    assert lib.pssgp_tune_set(3, old) == 0


def test_noalloc_size_limits_stated_in_the_header(lib):
    """The allocation-free log-likelihood accepts n while the workspace of the
    scan plan fits its 32 MiB scratch; the header states the resulting limits
    per state dimension, which must be the largest n with
    pssgp_workspace_size(d, n) <= 32 MiB (sizes are non-decreasing in n)."""
    text = " ".join(open(os.path.join(ROOT, "include", "pssgp.h")).read().replace("*", " ").split())
    for d in (1, 2, 3, 6, 8):
        lo, hi = 1, 1 << 22
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if lib.pssgp_workspace_size(d, mid) <= 32 << 20:
                lo = mid
            else:
                hi = mid - 1
        assert f"{lo:,} at d = {d}" in text, (d, lo)


def test_step_count_bound(lib):
    """n above 2^40 is rejected (keeps every workspace size far from int64
    overflow)."""
    assert lib.pssgp_workspace_size(6, 1 << 40) > 0
    assert lib.pssgp_workspace_size(6, (1 << 40) + 1) == 0
    assert lib.pssgp_workspace_size_grad(6, (1 << 41)) == 0


def test_split_series_argument_errors(lib):
    """The split-series calls reject bad arguments on the host before any
    launch (dummy pointers are never dereferenced); the gradient mode of the
    filter calls asks for the gradient's workspace."""
    import ctypes
    fake = ctypes.c_void_p(256)
    mm = P.build_model("rbf", 1.0, 1.0)
    m = ctypes.byref(mm.raw)
    EINVAL, EWS = -1, -4
    nan, inf = float("nan"), float("inf")
    assert lib.pssgp_split_agg_doubles(6, 0) == 2 * 36 + 18 and lib.pssgp_split_agg_doubles(6, 1) == 36 + 6 + 21
    assert lib.pssgp_split_agg_doubles(0, 0) == 0 and lib.pssgp_split_agg_doubles(9, 1) == 0
    n = 1000
    big = 1 << 34
    small_grad = lib.pssgp_workspace_size(6, n)
    assert lib.pssgp_workspace_size_grad(6, n) > small_grad
    red = lambda *a: lib.pssgp_split_filter_reduce(m, fake, fake, fake, fake, 0, *a)
    assert red(n, nan, nan, 3, fake, fake, big, None) == EINVAL            # mode outside 0..2
    assert red(n, inf, nan, 1, fake, fake, big, None) == EINVAL            # an infinite boundary time
    assert red(n, nan, -inf, 1, fake, fake, big, None) == EINVAL
    assert red(0, nan, nan, 1, fake, fake, big, None) == EINVAL            # empty chunk
    assert red(n, nan, nan, 1, None, fake, big, None) == EINVAL            # no output
    assert red(n, nan, nan, 2, fake, fake, small_grad, None) == EWS        # gradient mode: gradient workspace
    fin = lambda *a: lib.pssgp_split_filter_finish(m, fake, fake, fake, fake, 0, *a)
    assert fin(n, nan, 1, fake, 2, 2, None, None, n, None, fake, big, None) == EINVAL   # rank >= G
    assert fin(n, nan, 1, fake, 0, 0, None, None, n, None, fake, big, None) == EINVAL   # G < 1
    assert fin(n, nan, 1, None, 2, 0, None, None, n, None, fake, big, None) == EINVAL   # no aggregates
    assert fin(n, nan, 1, fake, 2, 0, fake, None, n - 1, None, fake, big, None) == EINVAL   # ld < n
    assert fin(n, nan, 2, fake, 2, 0, None, None, n, None, fake, small_grad, None) == EWS
    assert lib.pssgp_split_smooth_reduce(m, 0, fake, fake, big, None) == EINVAL
    assert lib.pssgp_split_smooth_finish(m, n, n, fake, 3, 3, None, None, None, None, fake, big, None) == EINVAL
    assert lib.pssgp_split_grad_mean_reduce(m, n, None, fake, big, None) == EINVAL
    assert lib.pssgp_split_grad_mean_reduce(m, n, fake, fake, small_grad, None) == EWS
    assert lib.pssgp_split_grad_mean_finish(m, n, fake, 2, 2, fake, fake, big, None) == EINVAL
    assert lib.pssgp_split_grad_mean_finish(m, n, fake, 2, 1, None, fake, big, None) == EINVAL
    assert lib.pssgp_split_grad_finish(m, None, 0, n, fake, 2, 1, fake, fake, big, None) == EINVAL   # no R
    assert lib.pssgp_split_grad_finish(m, fake, 0, n, fake, 2, 1, None, fake, big, None) == EINVAL   # no grad
    assert lib.pssgp_split_grad_finish(m, fake, 0, n, fake, 2, -1, fake, fake, big, None) == EINVAL
    assert lib.pssgp_split_grad_finish(m, fake, 0, n, fake, 2, 1, fake, fake, small_grad, None) == EWS
