"""GPU parity of the batched log-likelihood (many independent series in one
pass) against the sequential oracle, series by series.

Each series s is filtered by the oracle with the model built directly at its
own (lengthscale, variance) and its own noise variance; the CUDA path uses one
model of the family, rescaled per series on the device.  Tolerance semantics
as in test_gpu_parity: |dl| <= tol * max(|l|, n_obs).
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


def oracle_loglik(kind, t, y, mask, ell, s2, R):
    if t.size == 0:
        return 0.0
    return oracle.run(om.make_model(kind, ell, s2), t, y, mask, R).loglik


def run_batched(kind, bt, mask=None, ell0=1.0, s20=1.0):
    m = P.build_model(kind, ell0, s20)
    n = bt.t.size
    mask = np.ones(n, np.uint8) if mask is None else mask
    ll, ws = P.loglik_batched(m, dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y),
                              dev(mask, torch.uint8))
    return ll.cpu().numpy(), P.status(ws)


def check_series(kind, bt, ll, mask=None, idx=None):
    idx = range(bt.B) if idx is None else idx
    worst = 0.0
    for s in idx:
        a, b = bt.offsets[s], bt.offsets[s + 1]
        ms = np.ones(b - a, np.uint8) if mask is None else mask[a:b]
        ref = oracle_loglik(kind, bt.t[a:b], bt.y[a:b], ms, bt.lengthscale[s], bt.variance[s], bt.noise[s])
        nobs = int(ms.sum())
        err = abs(ll[s] - ref) / max(abs(ref), nobs, 1)
        assert err <= TOL[kind], (kind, s, b - a, ll[s], ref, err)
        worst = max(worst, err)
    return worst


# lengths: empty, single-step, shorter than a warp, tile-ragged, long
LENGTHS = [0, 1, 2, 7, 31, 33, 0, 257, 1000, 4099, 1, 12_345, 3, 65_536]


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf", "matern12"])
def test_batched_matches_oracle_per_series(kind):
    bt = wl.series_batch(seed=11, lengths=LENGTHS)
    bt.variance[:] = np.exp(np.random.default_rng(5).uniform(np.log(0.3), np.log(3.0), bt.B))
    ll, st = run_batched(kind, bt)
    assert st == 0
    check_series(kind, bt, ll)


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_batched_model_built_elsewhere(kind):
    """The family's model may be built at any (lengthscale, variance): the
    per-series rescaling is relative to where it was built."""
    bt = wl.series_batch(seed=12, lengths=[500, 2000, 77, 9000])
    ll, st = run_batched(kind, bt, ell0=0.37, s20=2.5)
    assert st == 0
    check_series(kind, bt, ll)


def test_batched_missing_measurements():
    bt = wl.series_batch(seed=13, lengths=[300, 5000, 1, 40, 2500])
    rng = np.random.default_rng(14)
    mask = (rng.uniform(size=bt.t.size) > 0.2).astype(np.uint8)
    a, b = bt.offsets[3], bt.offsets[4]
    mask[a:b] = 0                               # one series fully missing: loglik 0
    ll, st = run_batched("matern52", bt, mask)
    assert st == 0
    assert ll[3] == 0.0
    check_series("matern52", bt, ll, mask)


def test_batched_equals_single_series_calls():
    """Cross-check against the single-series entry point on the same device."""
    bt = wl.series_batch(seed=15, lengths=[3000, 20_000, 150, 8000])
    ll, st = run_batched("matern32", bt)
    assert st == 0
    for s in range(bt.B):
        t, y = bt.series(s)
        m = P.build_model("matern32", bt.lengthscale[s], bt.variance[s])
        l1, ws = P.loglik(m, dev(t), dev(y), dev(np.ones(t.size, np.uint8), torch.uint8), bt.noise[s])
        ref = float(l1.cpu().numpy()[0])
        assert abs(ll[s] - ref) <= 1e-11 * max(abs(ref), t.size)


def test_batched_more_series_than_steps():
    """Many empty series: every offset is still checked, empty series get 0."""
    bt = wl.series_batch(seed=16, lengths=[0, 0, 1, 0, 2, 0, 0, 0, 3, 0])
    ll, st = run_batched("matern32", bt)
    assert st == 0
    check_series("matern32", bt, ll)
    assert np.all(ll[[0, 1, 3, 5, 6, 7, 9]] == 0.0)


def test_batched_status_flags():
    bt = wl.series_batch(seed=17, lengths=[100, 200, 300])
    m = P.build_model("matern32", 1.0, 1.0)
    args = (dev(bt.t), dev(bt.y), dev(np.ones(bt.t.size, np.uint8), torch.uint8))
    bad = bt.params().copy()
    bad[1, 0] = -1.0                            # non-positive lengthscale
    ll, ws = P.loglik_batched(m, dev(bt.offsets, torch.int64), dev(bad), *args)
    assert P.status(ws) & P.EBATCH
    off = bt.offsets.copy()
    off[1], off[2] = off[2], off[1]             # decreasing offsets
    ll, ws = P.loglik_batched(m, dev(off, torch.int64), dev(bt.params()), *args)
    assert P.status(ws) & P.EBATCH
    off = bt.offsets.copy()
    off[-1] -= 1                                # offsets[B] != n
    ll, ws = P.loglik_batched(m, dev(off, torch.int64), dev(bt.params()), *args)
    assert P.status(ws) & P.EBATCH


def test_batched_deterministic():
    bt = wl.series_batch(seed=18, lengths=[40_000, 123, 7777, 31_000])
    a, _ = run_batched("rbf", bt)
    b, _ = run_batched("rbf", bt)
    assert np.array_equal(a, b)


def test_batched_full_size_sampled():
    """The 4,096-series workload (about 63 M steps, Matern-3/2 and 5/2 mixed)
    run as one call per family, in the launch configuration of the benchmark;
    a sample of series (shortest, longest and random ones) against the oracle."""
    bt = wl.series_batch(**wl.BATCH)
    kinds = np.array(bt.kind)
    lens = np.diff(bt.offsets)
    rng = np.random.default_rng(19)
    for kind in ("matern32", "matern52"):
        idx = np.flatnonzero(kinds == kind)
        sub = wl.subset(bt, idx)
        ll, st = run_batched(kind, sub)
        assert st == 0
        assert np.all(np.isfinite(ll))
        sl = lens[idx]
        pick = sorted({int(np.argmin(sl)), int(np.argmax(sl)), *rng.choice(idx.size, 4, replace=False).tolist()})
        check_series(kind, sub, ll, idx=pick)


@pytest.mark.parametrize("warps", [4, 8, 12, 16])
def test_batched_every_tuning(warps):
    """Every lane count the autotuner may pick gives the oracle's results."""
    bt = wl.series_batch(seed=20, lengths=[70_000, 5, 33_333, 129, 100_000, 1])
    saved = P.tune_get(3)
    try:
        P.tune_set(3, warps)
        ll, st = run_batched("matern52", bt)
    finally:
        P.tune_set(3, saved)
    assert st == 0
    check_series("matern52", bt, ll)


def test_autotune_keeps_results():
    bt = wl.series_batch(seed=21, lengths=[50_000, 20_000, 90_000, 3])
    m = P.build_model("matern32", 1.0, 1.0)
    args = (dev(bt.offsets, torch.int64), dev(bt.params()), dev(bt.t), dev(bt.y),
            dev(np.ones(bt.t.size, np.uint8), torch.uint8))
    saved = P.tune_get(2)
    try:
        w, ms = P.autotune_loglik_batched(m, *args, reps=2)
        assert w in (4, 8, 12, 16) and ms > 0.0
        assert P.tune_get(2) == w
        ll, ws = P.loglik_batched(m, *args)
    finally:
        P.tune_set(2, saved)
    assert P.status(ws) == 0
    check_series("matern32", bt, ll.cpu().numpy())


def test_graph_replay_with_new_parameters():
    """Both families of a mixed batch recorded into one CUDA graph; the
    per-series parameters are device data, so a replay after updating them
    in place gives the new log-likelihoods (bit-identical to direct calls)."""
    bt = wl.series_batch(seed=22, B=24, n_min=1000, n_max=20_000)
    kinds = np.array(bt.kind)
    parts = []
    for kind in ("matern32", "matern52"):
        sub = wl.subset(bt, np.flatnonzero(kinds == kind))
        m = P.build_model(kind, 1.0, 1.0)
        d = dict(m=m, sub=sub, off=dev(sub.offsets, torch.int64), par=dev(sub.params()), t=dev(sub.t),
                 y=dev(sub.y), mask=dev(np.ones(sub.t.size, np.uint8), torch.uint8))
        d["ws"] = P.workspace(m.d, sub.t.size, torch.device("cuda"))
        d["ll"] = torch.full((sub.B,), float("nan"), dtype=torch.float64, device="cuda")
        P.loglik_batched(d["m"], d["off"], d["par"], d["t"], d["y"], d["mask"], ws=d["ws"], out=d["ll"])  # warm-up
        parts.append((kind, d))
    torch.cuda.synchronize()
    g = P.Graph()
    with g:
        for _, d in parts:
            P.loglik_batched(d["m"], d["off"], d["par"], d["t"], d["y"], d["mask"], ws=d["ws"], out=d["ll"])
    for scale in (1.0, 1.7):
        for _, d in parts:
            d["par"][:, 0] = torch.as_tensor(d["sub"].lengthscale * scale, device="cuda")
        g.launch()
        torch.cuda.synchronize()
        for kind, d in parts:
            got = d["ll"].cpu().numpy().copy()
            ref, _ = P.loglik_batched(d["m"], d["off"], d["par"], d["t"], d["y"], d["mask"])
            assert np.array_equal(got, ref.cpu().numpy())
            sub = wl.subset(d["sub"], np.arange(d["sub"].B))
            sub.lengthscale = sub.lengthscale * scale
            check_series(kind, sub, got, idx=[0, sub.B - 1])


@pytest.mark.parametrize("kind", ["matern32", "matern52"])
def test_failed_series_are_nan_and_leave_the_others_intact(kind):
    """A series with a NaN observation, one with a non-positive lengthscale
    and one whose times decrease, inside a batch of healthy series: the three
    get NaN log-likelihoods and gradients, the status word carries their bits,
    and every healthy series (including those after the bad ones in the flat
    scan) still matches the oracle."""
    bt = wl.series_batch(seed=45, lengths=[3000, 2500, 4000, 1800, 2200, 5000, 700], kinds=(kind,))
    params = bt.params().copy()
    t, y = bt.t.copy(), bt.y.copy()
    y[bt.offsets[1] + 100] = np.nan                    # series 1: a non-finite observation
    params[3, 0] = -1.0                                # series 3: a negative lengthscale
    a4 = bt.offsets[4]
    t[a4 + 50] = t[a4 + 49] - 1.0                      # series 4: the times decrease
    bad = {1, 3, 4}
    m = P.build_model(kind, 1.0, 1.0)
    n = t.size
    args = (dev(bt.offsets, torch.int64), dev(params), dev(t), dev(y), dev(np.ones(n, np.uint8), torch.uint8))
    ll, ws = P.loglik_batched(m, *args)
    st = P.status(ws)
    assert st & P.ENAN and st & P.EBATCH and st & P.EUNSORTED
    llg, g, wsg = P.loglik_grad_batched(m, *args)
    stg = P.status(wsg)
    assert stg & P.ENAN and stg & P.EBATCH and stg & P.EUNSORTED
    ll, llg, g = ll.cpu().numpy(), llg.cpu().numpy(), g.cpu().numpy()
    for s in range(bt.B):
        if s in bad:
            assert np.isnan(ll[s]) and np.isnan(llg[s]) and np.all(np.isnan(g[s])), s
            continue
        a, b = bt.offsets[s], bt.offsets[s + 1]
        rll, rg, sc = oracle.loglik_grad_fwd(kind, bt.lengthscale[s], bt.variance[s], t[a:b], y[a:b],
                                             np.ones(b - a, np.uint8), bt.noise[s], with_scale=True)
        assert abs(ll[s] - rll) <= TOL[kind] * max(abs(rll), b - a), (s, ll[s], rll)
        assert abs(llg[s] - rll) <= TOL[kind] * max(abs(rll), b - a), (s, llg[s], rll)
        floor = np.maximum(sc / np.sqrt(b - a), 1e-5 * np.sqrt(b - a))
        assert np.max(np.abs(g[s] - rg) / np.maximum(np.abs(rg), floor)) <= 1e-8, (s, g[s], rg)


def test_batched_prior_workload_sampled():
    """The benchmark's 4,096-series workload with y drawn from the prior
    (the library's simulation, seeds as in the benchmark), one call per
    family.  The sampled series are replaced in the batch by the oracle's own
    simulation of them (the same Philox4x32-10 stream: the two simulations
    agree to about 1e-10, which smooth, nearly noise-free series amplify in
    the log-likelihood), so that the GPU and the oracle evaluate the same
    inputs."""
    offs, kinds, params = wl.prior_batch_spec(**wl.PRIOR_BATCH)
    kinds = np.array(kinds)
    rng = np.random.default_rng(46)
    for fi, kind in enumerate(("matern32", "matern52")):
        off, par = wl.subset_spec(offs, params, np.flatnonzero(kinds == kind))
        m = P.build_model(kind, 1.0, 1.0)
        offd = dev(off, torch.int64)
        seed = 300 + fi
        t, y, st = P.simulate_prior(m, offd, dev(par), seed=seed)
        assert int(st.item()) == 0
        lens = np.diff(off)
        pick = sorted({int(np.argmin(lens)), int(np.argmax(lens)), *rng.choice(lens.size, 2, replace=False).tolist()})
        ref = {}
        t, y = t.clone(), y.clone()
        for s in pick:
            n = int(lens[s])
            mo = om.make_model(kind, par[s, 0], par[s, 1])
            rt, ry = oracle.simulate_series(mo, par[s, 2], n, seed, s)
            a = int(off[s])
            t[a:a + n] = dev(rt)
            y[a:a + n] = dev(ry)
            ref[s] = oracle.run(mo, rt, ry, np.ones(n, np.uint8), par[s, 2]).loglik
        ll, ws = P.loglik_batched(m, offd, dev(par), t, y, torch.ones(t.numel(), dtype=torch.uint8, device="cuda"))
        assert P.status(ws) == 0
        ll = ll.cpu().numpy()
        assert np.all(np.isfinite(ll))
        for s in pick:
            n = int(lens[s])
            assert abs(ll[s] - ref[s]) <= TOL[kind] * max(abs(ref[s]), n), (kind, s, ll[s], ref[s])
