"""GPU parity of the batched prediction (pssgp_predict_batched): B series,
each with its own training and prediction times and hyperparameters, merged,
filtered and smoothed in one pass.  Every series is checked against the
oracle's sequential prediction (merge of Sec. 4.3, Kalman filter, RTS
smoother) at that series' own hyperparameters, at the parity tolerances of
the single-series tests (1e-9 Matern, 1e-6 RBF-6; mean relative to
max(|m|, sqrt(v)), variance relative, log-likelihood relative to
max(|ll|, n_obs))."""
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


def make_batch(seed, n_train, n_test, kind_ell=(0.3, 3.0), ties=True):
    """Series s: n_train[s] sorted training times on [0, 0.01 n] with a
    two-tone y, n_test[s] prediction times spread over a slightly wider
    range (before the first and after the last training time too), some of
    them equal to training times."""
    rng = np.random.default_rng(seed)
    tt, yy, ts = [], [], []
    for nt, nu in zip(n_train, n_test):
        span = 0.01 * max(nt + nu, 10)
        t = np.sort(rng.uniform(0.0, span, nt))
        y = np.sin(3.0 * t) + 0.5 * np.sin(11.0 * t) + rng.normal(0.0, 0.1, nt)
        u = np.sort(rng.uniform(-0.1 * span, 1.1 * span, nu))
        if ties and nt > 0 and nu > 2:
            u[nu // 2] = t[nt // 2]
            u = np.sort(u)
        tt.append(t); yy.append(y); ts.append(u)
    toff = np.concatenate([[0], np.cumsum([len(t) for t in tt])]).astype(np.int64)
    uoff = np.concatenate([[0], np.cumsum([len(u) for u in ts])]).astype(np.int64)
    B = len(n_train)
    params = np.stack([np.exp(rng.uniform(*np.log(kind_ell), B)), np.exp(rng.uniform(np.log(0.5), np.log(2.0), B)),
                       np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), B))], axis=1)
    cat = lambda xs: np.concatenate(xs) if sum(len(x) for x in xs) else np.empty(0)
    return toff, uoff, params, cat(tt), cat(yy), cat(ts)


def run_batched(kind, toff, uoff, params, t, y, u, order=6):
    m = P.build_model(kind, 1.0, 1.0, order=order)
    mean, var, ll, ws = P.predict_batched(m, dev(toff, torch.int64), dev(uoff, torch.int64), dev(params), dev(t),
                                          dev(y), dev(u))
    st = P.status(ws)
    return mean.cpu().numpy(), var.cpu().numpy(), ll.cpu().numpy(), st


def check_series(kind, s, toff, uoff, params, t, y, u, mean, var, ll, report, what, order=6):
    a, b = toff[s], toff[s + 1]
    c, d = uoff[s], uoff[s + 1]
    if b == a and d == c:                     # an empty series: log-likelihood 0, no outputs
        assert ll[s] == 0.0
        return 0.0
    o = om.make_model(kind, params[s, 0], params[s, 1], order=order)
    fm, fv, res, _ = oracle.predict(o, t[a:b], y[a:b], u[c:d], params[s, 2])
    tol = TOL[kind]
    em = np.max(np.abs(mean[c:d] - fm) / np.maximum(np.abs(fm), np.sqrt(fv))) if d > c else 0.0
    ev = np.max(np.abs(var[c:d] - fv) / fv) if d > c else 0.0
    el = abs(ll[s] - res.loglik) / max(abs(res.loglik), b - a, 1)
    worst = max(em, ev, el)
    assert np.isfinite(worst) and worst <= tol, (what, s, em, ev, el)
    return worst


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_batched_prediction_equals_oracle_per_series(kind, report):
    n_train = [0, 1, 2, 37, 500, 3000, 7, 1200, 64, 0, 2049, 5]
    n_test = [3, 0, 1, 5, 100, 31, 0, 250, 64, 0, 17, 40]
    toff, uoff, params, t, y, u = make_batch(71, n_train, n_test)
    mean, var, ll, st = run_batched(kind, toff, uoff, params, t, y, u)
    assert st == 0
    worst = 0.0
    for s in range(len(n_train)):
        worst = max(worst, check_series(kind, s, toff, uoff, params, t, y, u, mean, var, ll, report, kind))
    report(f"batched prediction vs oracle per series, {kind} (tol {TOL[kind]:g})", worst, TOL[kind])
    assert ll[9] == 0.0                       # an empty series


def test_batched_prediction_equals_single_series_calls(report):
    """Each series of the batch against pssgp_predict on that series alone
    (the same kernels on a different concatenation: rounding only)."""
    n_train = [800, 1, 4000, 33, 0, 129]
    n_test = [80, 2, 10, 1, 7, 0]
    toff, uoff, params, t, y, u = make_batch(72, n_train, n_test)
    mean, var, ll, st = run_batched("matern52", toff, uoff, params, t, y, u)
    assert st == 0
    worst = 0.0
    for s in range(len(n_train)):
        a, b, c, d = toff[s], toff[s + 1], uoff[s], uoff[s + 1]
        if b == a or d == c:
            continue
        m = P.build_model("matern52", params[s, 0], params[s, 1])
        m1, v1, l1, ws = P.predict(m, dev(t[a:b]), dev(y[a:b]), dev(u[c:d]), params[s, 2])
        assert P.status(ws) == 0
        m1, v1, l1 = m1.cpu().numpy(), v1.cpu().numpy(), float(l1.item())
        worst = max(worst, np.max(np.abs(mean[c:d] - m1) / np.maximum(np.abs(m1), np.sqrt(v1))),
                    np.max(np.abs(var[c:d] - v1) / v1), abs(ll[s] - l1) / max(abs(l1), b - a))
    report("batched prediction vs single-series pssgp_predict", worst, 1e-11)
    assert worst <= 1e-11


def test_failed_series_are_nan_and_leave_the_others_intact():
    """A non-positive lengthscale, a NaN observation, decreasing training
    times and a NaN prediction time, each in its own series of a batch: those
    four get NaN outputs; every other series matches the oracle."""
    n_train = [300, 200, 250, 180, 220, 260, 150]
    n_test = [20, 15, 25, 10, 30, 12, 18]
    toff, uoff, params, t, y, u = make_batch(73, n_train, n_test, ties=False)
    params = params.copy(); t = t.copy(); y = y.copy(); u = u.copy()
    params[1, 0] = -1.0                                  # series 1: bad lengthscale
    y[toff[3] + 50] = np.nan                             # series 3: NaN observation
    a = toff[4]
    t[a + 10], t[a + 11] = t[a + 11], t[a + 10]          # series 4: decreasing training times
    u[uoff[5] + 3] = np.nan                              # series 5: NaN prediction time
    mean, var, ll, st = run_batched("matern32", toff, uoff, params, t, y, u)
    assert st != 0
    for s in (1, 3, 4, 5):
        assert np.all(np.isnan(mean[uoff[s]:uoff[s + 1]])) and np.all(np.isnan(var[uoff[s]:uoff[s + 1]]))
        assert np.isnan(ll[s])
    for s in (0, 2, 6):
        check_series("matern32", s, toff, uoff, params, t, y, u, mean, var, ll, None, "healthy")


def test_batched_prediction_large_batch_sampled(report):
    """The 4,096-series batched workload's Matern-5/2 half (about 31 M
    training steps) with 1 % prediction times per series: sampled series
    against the oracle, and the batch's status clean."""
    bt = wl.series_batch(**wl.BATCH)
    idx = np.flatnonzero(np.array(bt.kind) == "matern52")
    sub = wl.subset(bt, idx)
    rng = np.random.default_rng(74)
    us, uo = [], [0]
    for s in range(sub.B):
        ts = sub.t[sub.offsets[s]:sub.offsets[s + 1]]
        k = max(1, (ts.size + 50) // 100)
        us.append(np.sort(rng.uniform(ts[0], ts[-1], k)))
        uo.append(uo[-1] + k)
    u = np.concatenate(us)
    uoff = np.array(uo, dtype=np.int64)
    mean, var, ll, st = run_batched("matern52", sub.offsets, uoff, sub.params(), sub.t, sub.y, u)
    assert st == 0
    worst = 0.0
    for s in rng.choice(sub.B, 12, replace=False):
        worst = max(worst, check_series("matern52", s, sub.offsets, uoff, sub.params(), sub.t, sub.y, u, mean, var,
                                        ll, report, "large"))
    report("batched prediction, 2,048-series Matern-5/2 batch, sampled series vs oracle", worst, 1e-9)


def test_batched_prediction_replays_from_a_cuda_graph():
    """The call captured once (P.Graph) and replayed gives the direct call's
    outputs bit for bit, also after the per-series parameters change in
    place between replays."""
    n_train = [400, 0, 900, 33]
    n_test = [40, 3, 9, 1]
    toff, uoff, params, t, y, u = make_batch(75, n_train, n_test)
    m = P.build_model("matern52", 1.0, 1.0)
    to, uo, pa = dev(toff, torch.int64), dev(uoff, torch.int64), dev(params)
    tt, yy, uu = dev(t), dev(y), dev(u)
    mean0, var0, ll0, ws = P.predict_batched(m, to, uo, pa, tt, yy, uu)
    assert P.status(ws) == 0
    ref = [(mean0.clone(), var0.clone(), ll0.clone())]
    mean, var, ll = torch.empty_like(mean0), torch.empty_like(var0), torch.empty_like(ll0)
    g = P.Graph()
    with g:
        P.predict_batched(m, to, uo, pa, tt, yy, uu, ws=ws, out=(mean, var, ll))
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(mean, ref[0][0]) and torch.equal(var, ref[0][1]) and torch.equal(ll, ref[0][2])
    pa.mul_(1.5)                                    # new hyperparameters, same buffers
    g.launch()
    torch.cuda.synchronize()
    m2, v2, l2, ws2 = P.predict_batched(m, to, uo, pa, tt, yy, uu)
    assert torch.equal(mean, m2) and torch.equal(var, v2) and torch.equal(ll, l2)
    assert not torch.equal(mean, ref[0][0])
