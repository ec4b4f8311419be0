"""GPU parity of the adjoint gradient of the log marginal likelihood with
respect to (log lengthscale, log variance, log noise variance) against the
oracle's forward-mode gradient (and, at the full 2^20-step size, also against
central differences of the oracle's log-likelihood).

Tolerance semantics, per component i: relative error
    |g_i - ref_i| / max(|ref_i|, s_i / sqrt(n_obs), 1e-5 sqrt(n_obs)) <= tol,
tol 1e-8 for Matern kernels and 1e-6 for the order-6 RBF Taylor model.
s_i is the sum over steps of |per-step term| of the forward-mode derivative
(the oracle returns it): a component is a sum of n_obs such terms, and
s_i / sqrt(n_obs) is the size of a sum of n_obs terms of that magnitude with
random signs.  A component below it (near an optimum, where the terms cancel)
is judged against that scale instead of its own value.  The per-step terms
are dimensionless; where every one of them is zero in exact arithmetic (the
lengthscale derivative of a one-observation series: H P_inf H^T does not
depend on the lengthscale) each still carries the rounding of the model's
tangent (up to ~1e-13 for the RBF model, whose tangent goes through a root
finder), so the scale is never taken below 1e-5 per sqrt(step).  Against central
differences (h = 1e-6): |g_i - fd_i| <= 1e-5 |fd_i| + 4 eps |loglik| / h, the
second term the rounding of the two log-likelihood values the difference
divides by 2h.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2102_09964_b300 as P
from oracle import model as om
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"matern12": 1e-8, "matern32": 1e-8, "matern52": 1e-8, "rbf": 1e-6}
# the log-likelihood itself: |d loglik| <= tol * max(|loglik|, n_obs)
LLTOL = {"matern12": 1e-9, "matern32": 1e-9, "matern52": 1e-9, "rbf": 1e-6}


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


@pytest.fixture(autouse=True)
def _rep(report):
    global REPORT
    REPORT = report


REPORT = None


def check_grad(g, ref, scale, nobs, tol, what=""):
    """Relative error per component, floored at max(scale / sqrt(n_obs), 1e-5 sqrt(n_obs))."""
    g = np.asarray(g, dtype=np.float64)
    floor = np.maximum(np.asarray(scale) / np.sqrt(max(nobs, 1)), 1e-5 * np.sqrt(max(nobs, 1)))
    err = np.max(np.abs(g - ref) / np.maximum(np.maximum(np.abs(ref), floor), 1e-300))
    if REPORT is not None:
        REPORT(f"gradient vs forward mode, {what[0] if isinstance(what, tuple) else what}".split("/")[0], err, tol)
    assert err <= tol, (what, g, ref, scale, err)
    return err


def fwd(kind, ell, s2, t, y, mask, R):
    return oracle.loglik_grad_fwd(kind, ell, s2, t, y, mask, R, with_scale=True)


def gpu_grad(kind, ell, s2, t, y, mask, R):
    m = P.build_model(kind, ell, s2)
    ll, g, ws = P.loglik_grad(m, dev(t), dev(y), dev(mask, torch.uint8), R)
    return float(ll.item()), g.cpu().numpy(), P.status(ws)


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
@pytest.mark.parametrize("n", [1, 2, 37, 3000, 40_001])
def test_grad_matches_forward_mode(kind, n):
    s = wl.random_series(31, max(n, 1), 0, T=n * 0.01 + 0.01)
    t, y = s.t_train, s.y_train
    rng = np.random.default_rng(32)
    mask = (rng.uniform(size=n) > 0.1).astype(np.uint8)
    ll, g, st = gpu_grad(kind, 0.7, 1.3, t, y, mask, 0.02)
    assert st == 0
    rll, rg, sc = fwd(kind, 0.7, 1.3, t, y, mask, 0.02)
    nobs = int(mask.sum())
    assert abs(ll - rll) <= LLTOL[kind] * max(abs(rll), nobs, 1)
    check_grad(g, rg, sc, nobs, TOL[kind], f"{kind}/{n}")


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_grad_long_gaps_ties_missing_runs(kind):
    s = wl.random_series(33, 6000, 0, T=60.0)
    t, y = s.t_train.copy(), s.y_train
    t[1000:] += 50.0                        # long step: halving/doubling path
    t[2000:2010] = t[2000]                  # ties (zero-length steps)
    t = np.maximum.accumulate(t)
    mask = np.ones(t.size, np.uint8)
    mask[3000:3500] = 0                     # a run of missing steps
    ll, g, st = gpu_grad(kind, 1.1, 0.9, t, y, mask, 0.05)
    assert st == 0
    rll, rg, sc = fwd(kind, 1.1, 0.9, t, y, mask, 0.05)
    check_grad(g, rg, sc, int(mask.sum()), TOL[kind], kind)


def test_grad_per_step_noise():
    s = wl.random_series(34, 5000, 0, T=50.0)
    R = np.exp(np.random.default_rng(35).uniform(np.log(1e-3), np.log(1e-1), 5000))
    mask = np.ones(5000, np.uint8)
    m = P.build_model("matern52", 0.8, 1.0)
    ll, g, ws = P.loglik_grad(m, dev(s.t_train), dev(s.y_train), dev(mask, torch.uint8), dev(R))
    assert P.status(ws) == 0
    rll, rg, sc = fwd("matern52", 0.8, 1.0, s.t_train, s.y_train, mask, R)
    check_grad(g.cpu().numpy(), rg, sc, 5000, TOL["matern52"], "matern52 per-step noise")


def test_grad_all_missing_is_zero():
    t = np.linspace(0.0, 10.0, 3000)
    ll, g, st = gpu_grad("matern32", 1.0, 1.0, t, np.zeros(3000), np.zeros(3000, np.uint8), 0.01)
    assert st == 0 and ll == 0.0 and np.all(np.abs(g) <= 1e-12)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_batched_grad_matches_forward_mode(kind):
    bt = wl.series_batch(seed=36, lengths=[0, 1, 2, 31, 33, 500, 4099, 0, 12_345, 3, 20_000])
    m = P.build_model(kind, 1.0, 1.0)
    mask = np.ones(bt.t.size, np.uint8)
    ll, g, ws = P.loglik_grad_batched(m, dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y),
                                      dev(mask, torch.uint8))
    assert P.status(ws) == 0
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    for s in range(bt.B):
        a, b = bt.offsets[s], bt.offsets[s + 1]
        if b == a:
            assert ll[s] == 0.0 and np.all(g[s] == 0.0)
            continue
        rll, rg, sc = fwd(kind, bt.lengthscale[s], bt.variance[s], bt.t[a:b], bt.y[a:b], mask[a:b],
                          bt.noise[s])
        assert abs(ll[s] - rll) <= LLTOL[kind] * max(abs(rll), b - a)
        check_grad(g[s], rg, sc, b - a, TOL[kind], (f"{kind} batched", s))


@pytest.mark.parametrize("kind", ["matern32", "matern52"])
def test_batched_grad_short_series_at_and_inside_chunk_starts(kind):
    """6,000 series of 1 to 3 steps with a quarter of the steps missing: at
    the default tuning every chunk holds a few steps, so series start at
    chunk starts and inside chunks, where the adjoint chunk aggregates reset
    (A = 0 after a series start)."""
    rng = np.random.default_rng(39)
    bt = wl.series_batch(seed=40, lengths=rng.integers(1, 4, size=6000), kinds=(kind,))
    m = P.build_model(kind, 1.0, 1.0)
    mask = (rng.uniform(size=bt.t.size) >= 0.25).astype(np.uint8)
    ll, g, ws = P.loglik_grad_batched(m, dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y),
                                      dev(mask, torch.uint8))
    assert P.status(ws) == 0
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    for s in rng.choice(bt.B, 400, replace=False):
        a, b = bt.offsets[s], bt.offsets[s + 1]
        nobs = max(int(mask[a:b].sum()), 1)
        rll, rg, sc = fwd(kind, bt.lengthscale[s], bt.variance[s], bt.t[a:b], bt.y[a:b], mask[a:b],
                          bt.noise[s])
        assert abs(ll[s] - rll) <= LLTOL[kind] * max(abs(rll), nobs)
        check_grad(g[s], rg, sc, nobs, TOL[kind], (f"{kind} batched short series", s))


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("R", [1e-6, 1e-9])
def test_grad_tiny_noise(kind, R):
    """Nearly noise-free data: J grows like 1/R in the chunk aggregates from
    which the adjoint chunk aggregates are formed (N = I + J P^-)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 16, M=0), 3_000)
    mask = np.ones(s.N, np.uint8)
    ll, g, st = gpu_grad(kind, 1.0, 1.0, s.t_train, s.y_train, mask, R)
    assert st == 0
    rll, rg, sc = fwd(kind, 1.0, 1.0, s.t_train, s.y_train, mask, R)
    assert abs(ll - rll) <= LLTOL[kind] * max(abs(rll), s.N)
    check_grad(g, rg, sc, s.N, TOL[kind], (f"{kind} tiny noise", R))


def test_batched_grad_full_size_sampled():
    """The 4,096-series workload, one call per family; sampled series against
    the oracle's forward-mode gradient."""
    bt = wl.series_batch(**wl.BATCH)
    kinds = np.array(bt.kind)
    lens = np.diff(bt.offsets)
    rng = np.random.default_rng(37)
    for kind in ("matern32", "matern52"):
        idx = np.flatnonzero(kinds == kind)
        sub = wl.subset(bt, idx)
        m = P.build_model(kind, 1.0, 1.0)
        ll, g, ws = P.loglik_grad_batched(m, dev(sub.offsets, torch.int64), dev(sub.params()), dev(sub.t),
                                          dev(sub.y), torch.ones(sub.t.size, dtype=torch.uint8, device="cuda"))
        assert P.status(ws) == 0
        ll, g = ll.cpu().numpy(), g.cpu().numpy()
        assert np.all(np.isfinite(g))
        sl = lens[idx]
        pick = sorted({int(np.argmin(sl)), int(np.argmax(sl)), *rng.choice(idx.size, 2, replace=False).tolist()})
        for s in pick:
            a, b = sub.offsets[s], sub.offsets[s + 1]
            rll, rg, sc = fwd(kind, sub.lengthscale[s], 1.0, sub.t[a:b], sub.y[a:b], np.ones(b - a, np.uint8),
                              sub.noise[s])
            check_grad(g[s], rg, sc, b - a, TOL[kind], (f"{kind} 4096-series batch", s))


def test_grad_full_size_rbf_vs_forward_mode_and_central_differences(report):
    """RBF-6 on the 2^20 training points, in the launch configuration of the
    benchmark, against the oracle's forward mode (relative 1e-6) and central
    differences (h = 1e-6) of its log-likelihood (relative 1e-5 plus the
    differences' rounding)."""
    from concurrent.futures import ThreadPoolExecutor
    s = wl.sinusoid_large()
    t, y = s.t_train, s.y_train
    mask = np.ones(t.size, np.uint8)
    ll, g, st = gpu_grad("rbf", 1.0, 1.0, t, y, mask, 0.01)
    assert st == 0
    # the oracle's three directions and the six difference points run in
    # threads (its C routines release the interpreter lock)
    m = om.make_model("rbf", 1.0, 1.0)
    with ThreadPoolExecutor(3) as ex:
        fw = list(ex.map(lambda p: oracle.loglik_tangent(m, t, y, mask, 0.01, p, with_scale=True),
                         oracle.GRAD_PARAMS))
    rll = fw[0][0]
    rg = np.array([f[1] for f in fw])
    sc = np.array([f[2] for f in fw])
    assert abs(ll - rll) <= LLTOL["rbf"] * max(abs(rll), t.size)
    check_grad(g, rg, sc, t.size, TOL["rbf"], "rbf 2^20")
    gfd = oracle.loglik_grad_fd("rbf", 1.0, 1.0, t, y, mask, 0.01, threads=6)
    noise = 4.0 * np.finfo(np.float64).eps * abs(rll) / 1e-6
    err = np.max(np.abs(g - gfd) / (1e-5 * np.abs(gfd) + noise))
    report("gradient vs central differences, rbf 2^20 (|d| / (1e-5|fd| + fd rounding))", err, 1.0)
    assert err <= 1.0, (g, gfd, noise)


def test_autograd_function_and_a_descent_step():
    bt = wl.series_batch(seed=38, lengths=[3000, 800, 15_000])
    m = P.build_model("matern52", 1.0, 1.0)
    off, t, y = dev(bt.offsets, torch.int64), dev(bt.t), dev(bt.y)
    mask = torch.ones(bt.t.size, dtype=torch.uint8, device="cuda")
    theta = torch.log(dev(bt.params())).requires_grad_(True)
    ll = P.batched_loglik(theta, m, off, t, y, mask)
    ll.sum().backward()
    _, g, _ = P.loglik_grad_batched(m, off, torch.exp(theta.detach()), t, y, mask)
    assert torch.equal(theta.grad, g)
    # a few Adam steps on the negative log-likelihood decrease it
    opt = torch.optim.Adam([theta], lr=0.05)
    first = None
    for _ in range(20):
        opt.zero_grad()
        loss = -P.batched_loglik(theta, m, off, t, y, mask).sum()
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    assert loss.item() < first


def test_grad_deterministic():
    s = wl.random_series(39, 30_000, 0, T=300.0)
    mask = np.ones(30_000, np.uint8)
    a = gpu_grad("rbf", 1.0, 1.0, s.t_train, s.y_train, mask, 0.01)[1]
    b = gpu_grad("rbf", 1.0, 1.0, s.t_train, s.y_train, mask, 0.01)[1]
    assert np.array_equal(a, b)
