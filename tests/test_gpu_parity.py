"""GPU parity: libpssgp (CUDA, sm_103a) against the sequential oracle on the
same seeded inputs, through the C ABI.

Tolerances: 1e-9 for Matern kernels, 1e-6 for the order-6 RBF Taylor model,
with these semantics: mean |dm| <= tol * max(|m|, sqrt(v)); variance
|dv| <= tol * v; log-likelihood |dl| <= tol * max(|l|, n_obs); filter states
entrywise relative to the state's own standard deviations.
"""
import math

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


def host(x):
    return x.detach().cpu().numpy()


REPORT = None


@pytest.fixture(autouse=True)
def _rep(report):
    global REPORT
    REPORT = report


def _rep_key(what):
    return str(what).split("/")[0]


def check_marginals(fm, fv, ll, rm, rv, rll, n_obs, tol, what=""):
    em = np.max(np.abs(fm - rm) / np.maximum(np.abs(rm), np.sqrt(rv)))
    ev = np.max(np.abs(fv - rv) / rv)
    el = abs(ll - rll) / max(abs(rll), n_obs) if ll is not None else 0.0
    if REPORT is not None:
        REPORT(f"posterior mean, {_rep_key(what)} (tol {tol:g})", em, tol)
        REPORT(f"posterior variance, {_rep_key(what)} (tol {tol:g})", ev, tol)
        if ll is not None:
            REPORT(f"log-likelihood, {_rep_key(what)} (tol {tol:g})", el, tol)
    assert np.isfinite(em) and np.isfinite(ev) and np.isfinite(el), (what, em, ev, el)
    assert em <= tol and ev <= tol and el <= tol, (what, em, ev, el)
    return em, ev, el


def check_states(x, Pk, rx, rP, tol, what=""):
    """x: (n, d), Pk: (n, d, d) vs oracle."""
    sd = np.sqrt(np.maximum(np.einsum("kii->ki", rP), 1e-300))
    ex = np.max(np.abs(x - rx) / np.maximum(np.abs(rx), sd))
    eP = np.max(np.abs(Pk - rP) / (sd[:, :, None] * sd[:, None, :]))
    if REPORT is not None:
        REPORT(f"state mean, {_rep_key(what)} (tol {tol:g})", ex, tol)
        REPORT(f"state covariance, {_rep_key(what)} (tol {tol:g})", eP, tol)
    assert np.isfinite(ex) and np.isfinite(eP), (what, ex, eP)
    assert ex <= tol and eP <= tol, (what, ex, eP)


def unpack(Pp, d):
    """packed (d(d+1)/2, n) -> (n, d, d)"""
    n = Pp.shape[1]
    out = np.empty((n, d, d))
    e = 0
    for i in range(d):
        for j in range(i, d):
            out[:, i, j] = Pp[e]
            out[:, j, i] = Pp[e]
            e += 1
    return out


def run_predict(kind, s, R, ell=1.0, s2=1.0):
    m = P.build_model(kind, ell, s2)
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), R)
    st = P.status(ws)
    return host(mean), host(var), float(host(ll)[0]), st


def oracle_predict(kind, s, R, ell=1.0, s2=1.0):
    o = om.make_model(kind, ell, s2)
    fm, fv, res, (t, y, mask, tp) = oracle.predict(o, s.t_train, s.y_train, s.t_test, R)
    return fm, fv, res, (t, y, mask, tp)


# --------------------------------------------------------------------------
# the fused prediction path
# --------------------------------------------------------------------------

def test_predict_small_workload():
    """1,000 training + 100 prediction points, Matern-3/2 (l = 0.5, s2 = 1, R = 0.01)."""
    s = wl.sinusoid_small()
    p = wl.SMALL
    mean, var, ll, st = run_predict(p["kind"], s, p["noise"], p["lengthscale"], p["variance"])
    assert st == 0
    fm, fv, res, _ = oracle_predict(p["kind"], s, p["noise"], p["lengthscale"], p["variance"])
    check_marginals(mean, var, ll, fm, fv, res.loglik, s.N, 1e-9, "small")


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
@pytest.mark.parametrize("n_train", [5_000, 150_001])
def test_predict_large_workload_prefix(kind, n_train):
    """Prefixes of the 2^20-point workload: many lanes and warps, ragged tails."""
    s = wl.prefix(wl.sinusoid_large(), n_train)
    mean, var, ll, st = run_predict(kind, s, 0.01)
    assert st == 0
    fm, fv, res, _ = oracle_predict(kind, s, 0.01)
    check_marginals(mean, var, ll, fm, fv, res.loglik, s.N, TOL[kind], f"{kind}/{n_train}")


class _tuning:
    """Scan tuning (warps per SM) for state dimension d inside the block."""

    def __init__(self, d, warps):
        self.d, self.warps = d, warps

    def __enter__(self):
        self.old = P.tune_get(self.d)
        P.tune_set(self.d, self.warps)

    def __exit__(self, *exc):
        P.tune_set(self.d, self.old)
        return False


@pytest.mark.parametrize("warps", [0, 2])
@pytest.mark.parametrize("kind", ["rbf", "matern52"])
def test_predict_full_size(kind, warps):
    """The full 2^20 + 10^4 workload in the launch configurations of the
    benchmark: one prediction at a time (the default tuning) and each of
    several concurrent predictions (2 warps per SM)."""
    s = wl.sinusoid_large()
    d = P.build_model(kind, 1.0, 1.0).d
    with _tuning(d, warps or P.tune_get(d)):
        mean, var, ll, st = run_predict(kind, s, 0.01)
    assert st == 0
    fm, fv, res, _ = oracle_predict(kind, s, 0.01)
    check_marginals(mean, var, ll, fm, fv, res.loglik, s.N, TOL[kind], f"full/{kind}/warps {warps or 'default'}")


@pytest.mark.parametrize("kind,order", [("rbf", 6), ("rbf", 4), ("matern52", 0)])
def test_predict_at_every_lane_tuning(kind, order):
    """1 to 8 warps per SM: the lane chunks change length (and, at d = 4..6,
    the prediction's reduce pass switches between its shared-memory and
    register warp scans at 4 warps per SM); every tuning must agree with the
    oracle and, to rounding, with the others."""
    s = wl.prefix(wl.sinusoid_large(), 150_001)
    o = om.make_model(kind, 1.0, 1.0, order=order) if order else om.make_model(kind, 1.0, 1.0)
    fm, fv, res, _ = oracle.predict(o, s.t_train, s.y_train, s.t_test, 0.01)
    m = P.build_model(kind, 1.0, 1.0, order=order) if order else P.build_model(kind, 1.0, 1.0)
    tol = TOL[kind]
    outs = []
    for warps in (1, 2, 3, 4, 8):
        with _tuning(m.d, warps):
            mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.01)
            assert P.status(ws) == 0
        mean, var, ll = host(mean), host(var), float(host(ll)[0])
        check_marginals(mean, var, ll, fm, fv, res.loglik, s.N, tol, f"tuning/{kind}{order or ''}/warps {warps}")
        outs.append((mean, var, ll))
    m0, v0, l0 = outs[3]
    for mean, var, ll in outs:
        assert np.max(np.abs(mean - m0) / np.maximum(np.abs(m0), np.sqrt(v0))) <= 1e-11
        assert np.max(np.abs(var - v0) / v0) <= 1e-11
        assert abs(ll - l0) <= 1e-12 * max(abs(l0), s.N)


# --------------------------------------------------------------------------
# filter, smoother, discretisation, merge as separate entry points
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n", [("matern32", 1100), ("matern52", 20_000), ("rbf", 20_000), ("matern12", 3000)])
def test_filter_and_smoother_states(kind, n):
    s = wl.prefix(wl.sinusoid_large(N=1 << 16, M=1000), n) if n > 1100 else wl.sinusoid_small()
    t, y, mask, tp = oracle.merge(s.t_train, s.y_train, s.t_test)
    o = om.make_model(kind, 1.0, 1.0)
    res = oracle.run(o, t, y, mask, 0.01)
    m = P.build_model(kind, 1.0, 1.0)
    d = m.d
    tg, yg, mg = dev(t), dev(y), dev(mask, torch.uint8)
    xf, Pf, ll, ws = P.filter(m, tg, yg, mg, 0.01)
    assert P.status(ws) == 0
    check_states(host(xf).T, unpack(host(Pf), d), res.m, res.P, TOL[kind], f"filter {kind}")
    assert abs(float(host(ll)[0]) - res.loglik) <= TOL[kind] * max(abs(res.loglik), s.N)
    fm, fv, xs, Ps, ws2 = P.smooth(m, tg, xf, Pf, states=True)
    assert P.status(ws2) == 0
    check_marginals(host(fm), host(fv), None, res.f_mean, res.f_var, None, s.N, TOL[kind], f"smooth {kind}")
    check_states(host(xs).T, unpack(host(Ps), d), res.ms, res.Ps, TOL[kind], f"smooth states {kind}")
    # the log-likelihood entry point sums per chunk from the fold's zero-start
    # terms (no propagate pass): the same value up to the summation order
    ll2, _ = P.loglik(m, tg, yg, mg, 0.01)
    assert abs(float(host(ll2)[0]) - float(host(ll)[0])) <= 1e-11 * max(abs(float(host(ll)[0])), s.N)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_discretize(kind):
    rng = np.random.default_rng(4)
    h = np.concatenate([rng.exponential(1e-3, 3000), [0.0, 0.0, 0.05, 0.3, 2.0, 17.0], rng.exponential(0.02, 500)])
    t = np.cumsum(h)
    o = om.make_model(kind, 1.0, 1.0)
    Fr, Qr = oracle.discretize(o, t)
    m = P.build_model(kind, 1.0, 1.0)
    d = m.d
    F, Q, ws = P.discretize(m, dev(t))
    assert P.status(ws) == 0
    F = host(F).T.reshape(-1, d, d)
    Q = unpack(host(Q), d)
    sF = np.abs(Fr).max(axis=(1, 2))
    sQ = np.abs(Qr).max(axis=(1, 2))
    assert np.max(np.abs(F - Fr).max(axis=(1, 2)) / np.maximum(sF, 1.0)) <= 1e-13
    nz = sQ > 0
    assert np.max(np.abs(Q - Qr).max(axis=(1, 2))[nz] / sQ[nz]) <= 1e-12
    assert np.all(np.abs(Q - Qr).max(axis=(1, 2))[~nz] == 0)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_discretize_entrywise_short_steps(kind):
    """Short steps (1e-6 to 3e-3 lengthscales) in warps that also hold a
    step of 17 lengthscales, so that every warp sums all stored Taylor terms
    of row 0: then every entry of Q at least 1e-12 of the step's largest
    agrees with the oracle (pinned entrywise against a 50-digit evaluation)
    to 1e-12 relative.  Rows 1..d-1 of Q come from row 0 through the
    Lyapunov identity on the device; this checks that they keep the relative
    accuracy of the small entries, which a normwise check does not see.  (With
    only short steps in a warp, its normwise term count leaves entries of
    order h^{2d-1} truncated: normwise negligible, not entrywise.)"""
    hk = np.zeros(64)                                   # two warps of steps k = 0..63
    long_k = [1, 33]
    rest = [k for k in range(1, 64) if k not in long_k]
    hk[long_k] = 17.0
    hk[rest] = np.logspace(-6, np.log10(3e-3), len(rest))
    t = np.cumsum(hk)
    o = om.make_model(kind, 1.0, 1.0)
    Fr, Qr = oracle.discretize(o, t)
    m = P.build_model(kind, 1.0, 1.0)
    d = m.d
    F, Q, ws = P.discretize(m, dev(t))
    assert P.status(ws) == 0
    Q = unpack(host(Q), d)
    worst = 0.0
    for k in range(1, t.size):
        if k in long_k:
            continue
        qmax = np.abs(Qr[k]).max()
        big = np.abs(Qr[k]) >= 1e-12 * qmax
        rel = np.abs(Q[k][big] - Qr[k][big]) / np.abs(Qr[k][big])
        worst = max(worst, rel.max())
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("seed", [0, 1])
def test_merge_bit_exact(seed):
    rng = np.random.default_rng(seed)
    tt = np.sort(np.round(rng.uniform(0, 50, 5000), 2))
    ts = np.sort(np.round(rng.uniform(0, 50, 1234), 2))      # many ties
    yy = rng.normal(size=tt.size)
    rt, ry, rm, rp = oracle.merge(tt, yy, ts)
    t, y, mask, tpos, ws = P.merge(dev(tt), dev(yy), dev(ts))
    assert P.status(ws) == 0
    np.testing.assert_array_equal(host(t), rt)
    np.testing.assert_array_equal(host(y), ry)
    np.testing.assert_array_equal(host(mask), rm)
    np.testing.assert_array_equal(host(tpos), rp)


# --------------------------------------------------------------------------
# the scan structure itself: level-0 chunk aggregates are the operator's fold
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_chunk_aggregates_are_operator_folds(kind):
    """Each lane's aggregate equals the fold of the Sec. 3 operator over the
    elements of its chunk (oracle operator, oracle elements)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 14, M=200), 3000)
    t, y, mask, tp = oracle.merge(s.t_train, s.y_train, s.t_test)
    o = om.make_model(kind, 1.0, 1.0)
    F, Q = oracle.discretize(o, t)
    A, b, C, eta, J = oracle.filter_elements(o, F, Q, y, mask, 0.01)
    m = P.build_model(kind, 1.0, 1.0)
    aggs, first, st = P.debug_filter_aggregates(m, dev(t), dev(y), dev(mask, torch.uint8), 0.01, lanes=128)
    assert st == 0
    n = t.size
    checked = 0
    for c, (k0, ag) in enumerate(zip(first, aggs)):
        k1 = first[c + 1] if c + 1 < len(first) else n
        if k1 <= k0 or c % 7:
            continue
        acc = (A[k0], b[k0], C[k0], eta[k0], J[k0])
        for k in range(k0 + 1, k1):
            acc = oracle.filter_combine(acc, (A[k], b[k], C[k], eta[k], J[k]))
        for u, v in zip(ag, acc):
            sc = max(np.abs(v).max(), 1e-300)
            assert np.abs(u - v).max() <= 1e-8 * sc + 1e-300, (c, np.abs(u - v).max(), sc)
        checked += 1
    assert checked >= 10


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,M", [(1, 0), (1, 1), (2, 0), (3, 5), (31, 2), (33, 1), (127, 7), (129, 0), (4097, 13)])
@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_small_and_ragged_sizes(N, M, kind):
    s = wl.random_series(100 + N + M, N, M, T=0.05 * (N + M) + 1.0)
    if M == 0:
        # predict needs M >= 0; compare the marginals at the training points via filter + smoother
        t, y, mask, tp = oracle.merge(s.t_train, s.y_train, s.t_test)
        o = om.make_model(kind, 0.7, 1.0)
        res = oracle.run(o, t, y, mask, 0.02)
        m = P.build_model(kind, 0.7, 1.0)
        xf, Pf, ll, ws = P.filter(m, dev(t), dev(y), dev(mask, torch.uint8), 0.02)
        fm, fv, _, _, _ = P.smooth(m, dev(t), xf, Pf)
        check_marginals(host(fm), host(fv), float(host(ll)[0]), res.f_mean, res.f_var, res.loglik, N, TOL[kind])
    else:
        mean, var, ll, st = run_predict(kind, s, 0.02, 0.7)
        assert st == 0
        fm, fv, res, _ = oracle_predict(kind, s, 0.02, 0.7)
        check_marginals(mean, var, ll, fm, fv, res.loglik, N, TOL[kind], f"{N}/{M}")


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
def test_long_gaps_ties_and_missing(kind):
    """Steps far beyond the longest Taylor step (halving + doubling path), duplicate times,
    long runs of missing measurements and per-step noise variances."""
    rng = np.random.default_rng(9)
    h = np.concatenate([rng.exponential(0.01, 2000), [0.0, 0.0, 3.0, 40.0, 0.0], rng.exponential(0.5, 300)])
    t = np.cumsum(h)
    mask = (rng.uniform(size=t.size) < 0.6).astype(np.uint8)
    mask[500:900] = 0
    y = (np.sin(t) + rng.normal(0, 0.1, t.size)) * mask
    R = rng.uniform(1e-3, 1e-1, t.size)
    o = om.make_model(kind, 0.8, 1.3)
    res = oracle.run(o, t, y, mask, R)
    m = P.build_model(kind, 0.8, 1.3)
    xf, Pf, ll, ws = P.filter(m, dev(t), dev(y), dev(mask, torch.uint8), dev(R))
    assert P.status(ws) == 0
    fm, fv, _, _, ws2 = P.smooth(m, dev(t), xf, Pf)
    assert P.status(ws2) == 0
    check_marginals(host(fm), host(fv), float(host(ll)[0]), res.f_mean, res.f_var, res.loglik, int(mask.sum()),
                    TOL[kind], "gaps")


def test_all_missing_is_prior():
    m = P.build_model("matern52", 1.0, 2.0)
    t = np.sort(np.random.default_rng(1).uniform(0, 30, 5000))
    xf, Pf, ll, ws = P.filter(m, dev(t), dev(np.zeros(t.size)), dev(np.zeros(t.size), torch.uint8), 0.01)
    fm, fv, _, _, _ = P.smooth(m, dev(t), xf, Pf)
    assert float(host(ll)[0]) == 0.0
    assert np.abs(host(fm)).max() == 0.0
    np.testing.assert_allclose(host(fv), 2.0, rtol=1e-12)


def test_status_flags_unsorted_and_nan():
    m = P.build_model("matern32", 1.0, 1.0)
    t = np.linspace(0, 1, 1000)
    t[500] = t[498]
    y = np.sin(t)
    _, _, _, ws = P.filter(m, dev(t), dev(y), dev(np.ones(1000), torch.uint8), 0.01)
    assert P.status(ws) & P.EUNSORTED
    t = np.linspace(0, 1, 1000)
    y[10] = np.nan
    _, _, _, ws = P.filter(m, dev(t), dev(y), dev(np.ones(1000), torch.uint8), 0.01)
    assert P.status(ws) & P.ENAN
    y[10] = 0.0
    _, _, _, ws = P.filter(m, dev(t), dev(y), dev(np.ones(1000), torch.uint8), 0.01)
    assert P.status(ws) == 0


def test_deterministic():
    s = wl.prefix(wl.sinusoid_large(), 50_000)
    a = run_predict("rbf", s, 0.01)
    b = run_predict("rbf", s, 0.01)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_concurrent_predictions_on_streams_equal_serial_ones():
    """Eight predictions of different series in flight on eight streams, each
    with its own workspace, at the benchmark's concurrent tuning (2 warps per
    SM): every result equals, bit for bit, the same prediction run alone on
    one stream (no state shared between calls)."""
    m = P.build_model("rbf", 1.0, 1.0)
    series = [wl.prefix(wl.sinusoid_large(seed=40 + i), 60_000 + 997 * i) for i in range(8)]
    ins = [(dev(s.t_train), dev(s.y_train), dev(s.t_test)) for s in series]
    with _tuning(m.d, 2):
        ref = []
        for tt, yy, ts in ins:
            mean, var, ll, ws = P.predict(m, tt, yy, ts, 0.01)
            assert P.status(ws) == 0
            ref.append((host(mean), host(var), float(host(ll)[0])))
        streams = [torch.cuda.Stream() for _ in ins]
        wss = [P.workspace(m.d, s.N + s.M) for s in series]
        outs = [None] * len(ins)
        cur = torch.cuda.current_stream()
        for rep in range(2):
            for i, ((tt, yy, ts), st) in enumerate(zip(ins, streams)):
                st.wait_stream(cur)
                with torch.cuda.stream(st):
                    outs[i] = P.predict(m, tt, yy, ts, 0.01, ws=wss[i])
            for st in streams:
                cur.wait_stream(st)
            torch.cuda.synchronize()
            for i, (mean, var, ll, ws) in enumerate(outs):
                assert P.status(ws) == 0
                np.testing.assert_array_equal(host(mean), ref[i][0])
                np.testing.assert_array_equal(host(var), ref[i][1])
                assert float(host(ll)[0]) == ref[i][2]
    fm, fv, res, _ = oracle_predict("rbf", series[3], 0.01)
    check_marginals(ref[3][0], ref[3][1], ref[3][2], fm, fv, res.loglik, series[3].N, TOL["rbf"], "concurrent/rbf")


def test_user_sde_with_scaled_measurement_row():
    """y = h0 x_0 + e with h0 = 2 (pssgp_model_from_sde): f = H x, so the
    marginals are those of the oracle run with the same H."""
    s = wl.sinusoid_small(N=400, M=40)
    o = om.make_model("matern32", 0.5, 1.0)
    o.H = 2.0 * o.H
    fm, fv, res, _ = oracle.predict(o, s.t_train, s.y_train, s.t_test, 0.01)
    m = P.model_from_sde(o.G, o.L, o.q, o.H)
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.01)
    assert P.status(ws) == 0
    check_marginals(host(mean), host(var), float(host(ll)[0]), fm, fv, res.loglik, s.N, 1e-9, "H = 2 e0")


def test_predict_from_host_buffers_equals_device_call():
    """pssgp_predict_host (host inputs and outputs, copies inside the call) on
    two streams gives the device call's results."""
    s = wl.prefix(wl.sinusoid_large(), 50_000)
    m = P.build_model("matern52", 1.0, 1.0)
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.01)
    ref = (host(mean), host(var), host(ll))
    ht = [torch.as_tensor(x).pin_memory() for x in (s.t_train, s.y_train, s.t_test)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [tuple(torch.full((k,), float("nan"), dtype=torch.float64).pin_memory() for k in (s.M, s.M, 1))
            for _ in streams]
    keep = [P.predict_host(m, *ht, 0.01, o, stream=st) for st, o in zip(streams, outs)]   # workspaces stay alive
    torch.cuda.synchronize()
    del keep
    for o in outs:
        assert np.array_equal(o[0].numpy(), ref[0]) and np.array_equal(o[1].numpy(), ref[1])
        assert o[2].numpy()[0] == ref[2][0]


@pytest.mark.parametrize("order", [2, 4, 8])
def test_predict_rbf_orders_up_to_the_largest_state(order):
    """RBF Taylor orders up to 8 (d = 8, the largest state dimension)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 15, M=400), 6000)
    m = P.build_model("rbf", 1.0, 1.0, order=order)
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.01)
    assert P.status(ws) == 0
    o = om.make_model("rbf", 1.0, 1.0, order=order)
    fm, fv, res, _ = oracle.predict(o, s.t_train, s.y_train, s.t_test, 0.01)
    check_marginals(host(mean), host(var), float(host(ll)[0]), fm, fv, res.loglik, s.N, 1e-6, f"rbf{order}")


def test_companion_drift_with_full_diffusion():
    """A companion drift whose white noise also drives the first states
    (L = (0.4, -0.3, 1)): F still takes the companion recursion, but Q has no
    rank-one structure on the last state, so every entry of Q is summed by
    its Taylor series instead of rows 1..d-1 following from row 0."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 15, M=400), 8000)
    o = om.make_model("matern52", 0.8, 1.0)
    o.L = np.array([[0.4], [-0.3], [1.0]])
    o.Pinf = om.lyapunov(o.G, o.W)
    m = P.model_from_sde(o.G, o.L, o.q, o.H)
    assert m.raw.companion == 1
    W = np.ctypeslib.as_array(m.raw.W)[:9].reshape(3, 3)
    assert np.count_nonzero(W) > 1
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.02)
    assert P.status(ws) == 0
    fm, fv, res, _ = oracle.predict(o, s.t_train, s.y_train, s.t_test, 0.02)
    check_marginals(host(mean), host(var), float(host(ll)[0]), fm, fv, res.loglik, s.N, 1e-9, "full W")


def _non_companion_sde():
    """Matern-5/2 in coordinates z = T^-1 x with T's first row e_0 (so
    H T = e_0^T) and the rest mixing: G' = T^-1 G T is not in companion form,
    the GP it defines is the same."""
    o = om.make_model("matern52", 0.7, 1.3)
    T = np.array([[1.0, 0.0, 0.0], [0.3, 1.0, -0.2], [0.5, 0.4, 1.0]])
    Ti = np.linalg.inv(T)
    return o, Ti @ o.G @ T, Ti @ o.L, o.H @ T


def test_non_companion_user_sde_predict():
    s = wl.prefix(wl.sinusoid_large(N=1 << 15, M=400), 8000)
    o, G, L, H = _non_companion_sde()
    m = P.model_from_sde(G, L, o.q, H, balance=False)
    assert m.raw.companion == 0
    mean, var, ll, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.02)
    assert P.status(ws) == 0
    fm, fv, res, _ = oracle.predict(o, s.t_train, s.y_train, s.t_test, 0.02)
    check_marginals(host(mean), host(var), float(host(ll)[0]), fm, fv, res.loglik, s.N, 1e-9, "user SDE")


def test_non_companion_user_sde_gradient():
    """The gradient of the rescaled family of the user SDE is the Matern
    family's gradient (the log-likelihood does not depend on coordinates)."""
    s = wl.prefix(wl.sinusoid_large(N=1 << 15, M=0), 6000)
    o, G, L, H = _non_companion_sde()
    m = P.model_from_sde(G, L, o.q, H, balance=False)
    mask = np.ones(s.N, np.uint8)
    ll, g, ws = P.loglik_grad(m, dev(s.t_train), dev(s.y_train), dev(mask, torch.uint8), 0.02)
    assert P.status(ws) == 0
    rll, rg = oracle.loglik_grad_fwd("matern52", 0.7, 1.3, s.t_train, s.y_train, mask, 0.02)
    assert abs(float(ll.item()) - rll) <= 1e-9 * max(abs(rll), s.N)
    assert np.max(np.abs(g.cpu().numpy() - rg) / np.maximum(np.abs(rg), s.N)) <= 1e-9
