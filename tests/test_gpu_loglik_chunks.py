"""The log-likelihood-only path against the library's propagate path and the
oracle.

Without per-step outputs, the log-likelihood is assembled per chunk: the
filter fold accumulates the log-likelihood of the chunk's observations given
the state 0 before it, and the chunk's term is then corrected with the filter
state before the chunk from the scan (a Gaussian integral, exact in exact
arithmetic).  pssgp_filter with per-step outputs still takes the propagate
pass (the sequential prediction-error sum inside each chunk), so the two are
compared directly, and both against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2102_09964_b300 as P
import workloads as wl
from oracle import model as om

pytestmark = pytest.mark.gpu

TOL = {"matern12": 1e-9, "matern32": 1e-9, "matern52": 1e-9, "rbf": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_09964_b300 import build
    build.build()
    P.lib()
    oracle.build()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def both_paths(kind, t, y, mask, R, ell=1.0, s2=1.0):
    m = P.build_model(kind, ell, s2)
    tg, yg, mg = dev(t), dev(y), dev(mask, torch.uint8)
    ll, ws = P.loglik(m, tg, yg, mg, R)
    assert P.status(ws) == 0
    _, _, llp, ws2 = P.filter(m, tg, yg, mg, R)          # per-step outputs: propagate pass
    assert P.status(ws2) == 0
    return float(ll.cpu()[0]), float(llp.cpu()[0])


def series(seed, n, offset=0.0, missing=0.2):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 0.01 * max(n, 1), n))
    y = offset + np.sin(3.0 * t) + 0.5 * np.sin(11.0 * t) + rng.normal(0.0, 0.1, n)
    mask = (rng.uniform(size=n) >= missing).astype(np.uint8)
    return t, y, mask


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
@pytest.mark.parametrize("n", [1, 7, 1000, 40_000, 300_000])
def test_loglik_path_equals_propagate_path(kind, n):
    t, y, mask = series(n + len(kind), n)
    ll, llp = both_paths(kind, t, y, mask, 0.01)
    assert abs(ll - llp) <= 1e-11 * max(abs(llp), int(mask.sum()), 1), (ll, llp)


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
def test_loglik_path_matches_oracle_offset_and_per_step_noise(kind):
    """A mean offset of 30 makes the zero-start terms large and the correction
    cancel most of them; per-step noise variances and 30 % missing steps."""
    n = 20_000
    t, y, mask = series(7, n, offset=30.0, missing=0.3)
    R = np.exp(np.random.default_rng(8).uniform(np.log(1e-3), np.log(1e-1), n))
    m = P.build_model(kind, 0.7, 2.0)
    ll, ws = P.loglik(m, dev(t), dev(y), dev(mask, torch.uint8), dev(R))
    assert P.status(ws) == 0
    ref = oracle.run(om.make_model(kind, 0.7, 2.0), t, y, mask, R).loglik
    assert abs(float(ll.cpu()[0]) - ref) <= TOL[kind] * max(abs(ref), int(mask.sum()))


@pytest.mark.parametrize("warps", [4, 16])
def test_loglik_path_across_lane_counts(warps):
    """Chunks of 1 to 60 steps: the same value from every tuning."""
    kind = "matern52"
    t, y, mask = series(11, 50_000)
    saved = P.tune_get(3)
    try:
        P.tune_set(3, warps)
        ll, llp = both_paths(kind, t, y, mask, 0.02)
    finally:
        P.tune_set(3, saved)
    ref = oracle.run(om.make_model(kind, 1.0, 1.0), t, y, mask, 0.02).loglik
    assert abs(ll - ref) <= 1e-9 * max(abs(ref), int(mask.sum()))
    assert abs(ll - llp) <= 1e-11 * max(abs(llp), int(mask.sum()))


def test_batched_short_series_at_and_inside_chunk_starts():
    """Series of 1 to 3 steps (some all-missing): at the default tuning every
    chunk holds a few steps, so series start both at chunk starts and inside
    chunks.  Every series against the oracle and against the gradient call,
    whose log-likelihood comes from the propagate pass."""
    rng = np.random.default_rng(21)
    lengths = rng.integers(1, 4, size=20_000)
    bt = wl.series_batch(seed=22, lengths=lengths, kinds=("matern52",))
    mask = (rng.uniform(size=bt.t.size) >= 0.25).astype(np.uint8)
    m = P.build_model("matern52", 1.0, 1.0)
    args = (m, dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y), dev(mask, torch.uint8))
    ll, ws = P.loglik_batched(*args)
    assert P.status(ws) == 0
    llg, _, ws2 = P.loglik_grad_batched(*args)
    assert P.status(ws2) == 0
    ll, llg = ll.cpu().numpy(), llg.cpu().numpy()
    nobs = np.add.reduceat(mask.astype(np.int64), bt.offsets[:-1])
    assert np.all(np.abs(ll - llg) <= 1e-11 * np.maximum(np.abs(llg), np.maximum(nobs, 1)))
    for s in rng.choice(bt.B, 1500, replace=False):
        a, b = bt.offsets[s], bt.offsets[s + 1]
        ms = mask[a:b]
        ref = oracle.run(om.make_model("matern52", bt.lengthscale[s], bt.variance[s]), bt.t[a:b], bt.y[a:b], ms,
                         bt.noise[s]).loglik
        assert abs(ll[s] - ref) <= 1e-9 * max(abs(ref), int(ms.sum()), 1), (s, ll[s], ref)


def test_batched_long_series_equal_single_calls():
    bt = wl.series_batch(seed=23, lengths=[70_000, 3, 1, 40_000, 9_999], kinds=("matern32",))
    m = P.build_model("matern32", 1.0, 1.0)
    n = bt.t.size
    ll, ws = P.loglik_batched(m, dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y),
                              dev(np.ones(n, np.uint8), torch.uint8))
    assert P.status(ws) == 0
    ll = ll.cpu().numpy()
    for s in range(bt.B):
        a, b = bt.offsets[s], bt.offsets[s + 1]
        ms = P.build_model("matern32", bt.lengthscale[s], bt.variance[s])
        one, w1 = P.loglik(ms, dev(bt.t[a:b]), dev(bt.y[a:b]), dev(np.ones(b - a, np.uint8), torch.uint8),
                           bt.noise[s])
        assert P.status(w1) == 0
        one = float(one.cpu()[0])
        assert abs(ll[s] - one) <= 1e-10 * max(abs(one), b - a)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("R", [1e-6, 1e-9])
def test_tiny_noise_prediction_and_loglik(kind, R):
    """Nearly noise-free data: J grows like 1/R in the chunk aggregates, and
    the closed forms solve with I + P J.  Prediction (closed-form smoother
    chunk aggregates) and both log-likelihood paths against the oracle at the
    usual tolerances (measured errors up to about 5e-11 at R = 1e-9)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 16, M=1000), 8_000)
    m = P.build_model(kind, 1.0, 1.0)
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), R)
    assert P.status(ws) == 0
    fm, fv, res, _ = oracle.predict(om.make_model(kind, 1.0, 1.0), s.t_train, s.y_train, s.t_test, R)
    mean, var, ll = mean.cpu().numpy(), var.cpu().numpy(), float(ll.cpu()[0])
    tol = TOL[kind]
    assert np.max(np.abs(mean - fm) / np.maximum(np.abs(fm), np.sqrt(fv))) <= tol
    assert np.max(np.abs(var - fv) / fv) <= tol
    assert abs(ll - res.loglik) <= tol * max(abs(res.loglik), s.N)
    t, y, mask, _ = oracle.merge(s.t_train, s.y_train, s.t_test)
    l2, w2 = P.loglik(m, dev(t), dev(y), dev(mask, torch.uint8), R)
    assert P.status(w2) == 0
    assert abs(float(l2.cpu()[0]) - res.loglik) <= tol * max(abs(res.loglik), s.N)
