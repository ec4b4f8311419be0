"""GPU parity of one long series split in time chunks (the pssgp_split_*
entry points and the exchange of paper_2102_09964_b300.split), with the ranks
run in lockstep on one GPU: every chunk's kernels run and finish before the
collectives are answered on the host, so no kernel waits on another.

Checked against the oracle's sequential filter and smoother over the whole
series (tolerances as the other parity tests: 1e-9 Matern, 1e-6 RBF-6) and
against the unsplit library calls.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2102_09964_b300 as P
import workloads as wl
from oracle import model as om
from paper_2102_09964_b300 import split

pytestmark = pytest.mark.gpu

TOL = {"matern32": 1e-9, "matern52": 1e-9, "rbf": 1e-6}


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


def merged(seed, n_train, n_test, T):
    s = wl.random_series(seed, n_train, n_test, T=T)
    return oracle.merge(s.t_train, s.y_train, s.t_test)[:3]


def run_split(m, t, y, mask, R, bounds, filter_outputs=False):
    G = len(bounds)
    chunks = [split.LibraryChunk(m, dev(t[a:b]), dev(y[a:b]), dev(mask[a:b], torch.uint8), R,
                                 filter_outputs=filter_outputs) for a, b in bounds]
    res = split.run_lockstep([split.chunk_protocol(c, r, G) for r, c in enumerate(chunks)])
    for c in chunks:
        assert P.status(c.ws) == 0
    fm = torch.cat([r[0] for r in res]).cpu().numpy()
    fv = torch.cat([r[1] for r in res]).cpu().numpy()
    lls = {float(r[2].item()) for r in res}
    assert len(lls) == 1
    return fm, fv, lls.pop(), chunks


def check(fm, fv, ll, rm, rv, rll, nobs, tol, report, what):
    em = np.max(np.abs(fm - rm) / np.maximum(np.abs(rm), np.sqrt(rv)))
    ev = np.max(np.abs(fv - rv) / rv)
    el = abs(ll - rll) / max(abs(rll), nobs)
    report(f"split series vs oracle: mean, {what} (tol {tol:g})", em, tol)
    report(f"split series vs oracle: variance, {what} (tol {tol:g})", ev, tol)
    report(f"split series vs oracle: log-likelihood, {what} (tol {tol:g})", el, tol)
    assert np.isfinite(em) and np.isfinite(ev) and np.isfinite(el)
    assert em <= tol and ev <= tol and el <= tol, (what, em, ev, el)


@pytest.mark.parametrize("kind", ["matern32", "matern52", "rbf"])
@pytest.mark.parametrize("G", [1, 2, 3, 4, 7])
def test_split_equals_oracle(kind, G, report):
    t, y, mask = merged(101, 20_000, 2_000, T=220.0)
    m = P.build_model(kind, 0.9, 1.2)
    fm, fv, ll, _ = run_split(m, t, y, mask, 0.02, split.chunk_bounds(t.size, G))
    res = oracle.run(om.make_model(kind, 0.9, 1.2), t, y, mask, 0.02)
    check(fm, fv, ll, res.f_mean, res.f_var, res.loglik, int(mask.sum()), TOL[kind], report, kind)


def test_uneven_chunks_at_missing_steps_and_across_a_long_gap(report):
    """Chunks of 1, 2 and 33 steps, a chunk that starts at a missing step,
    one that is a single missing step, a boundary across a gap of 40
    lengthscales (the transition there is the doubling path), and ties."""
    t, y, mask = merged(102, 6_000, 600, T=66.0)
    t = t.copy()
    t[3300:] += 40.0
    t[1000:1004] = t[1000]
    mask = mask.copy()
    mask[3300] = 0
    mask[5000] = 0
    bounds = [(0, 1), (1, 3), (3, 36), (36, 3300), (3300, 5000), (5000, 5001), (5001, t.size)]
    m = P.build_model("matern52", 1.0, 1.0)
    fm, fv, ll, _ = run_split(m, t, y, mask, 0.05, bounds)
    res = oracle.run(om.make_model("matern52", 1.0, 1.0), t, y, mask, 0.05)
    check(fm, fv, ll, res.f_mean, res.f_var, res.loglik, int(mask.sum()), 1e-9, report, "uneven chunks")


@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_split_filter_states_equal_the_unsplit_filter(kind, report):
    """The filter outputs of every chunk equal pssgp_filter's on the whole
    series (both in the library: the same elements, scans grouped
    differently), and the log-likelihood-only finishing call equals the one
    with outputs."""
    t, y, mask = merged(103, 30_000, 1_000, T=310.0)
    m = P.build_model(kind, 1.0, 1.0)
    xf, Pf, ll, ws = P.filter(m, dev(t), dev(y), dev(mask, torch.uint8), 0.01)
    assert P.status(ws) == 0
    xf, Pf = xf.cpu().numpy(), Pf.cpu().numpy()
    bounds = split.chunk_bounds(t.size, 3)
    _, _, lls, chunks = run_split(m, t, y, mask, 0.01, bounds, filter_outputs=True)
    d = m.d
    pidx = [(i, j) for i in range(d) for j in range(i, d)]
    diag = [e for e, (i, j) in enumerate(pidx) if i == j]
    sd = np.sqrt(np.maximum(Pf[diag], 1e-300))                  # (d, n): each state entry's own scale
    psc = np.array([sd[i] * sd[j] for i, j in pidx])            # (d(d+1)/2, n)
    worst = 0.0
    for (a, b), c in zip(bounds, chunks):
        dx = np.max(np.abs(c.xf.cpu().numpy() - xf[:, a:b]) / np.maximum(np.abs(xf[:, a:b]), sd[:, a:b]))
        dP = np.max(np.abs(c.Pf.cpu().numpy() - Pf[:, a:b]) / psc[:, a:b])
        worst = max(worst, dx, dP)
    report(f"split filter states vs unsplit library filter, {kind}", worst, 1e-9)
    assert worst <= 1e-9
    # log-likelihood only (no per-step outputs, no smoother): the chunk sums of reading r21
    tot = 0.0
    nan = float("nan")
    ends = [(nan if r == 0 else float(t[bounds[r - 1][1] - 1]), nan if r + 1 == len(bounds) else float(t[b]))
            for r, (a, b) in enumerate(bounds)]
    aggs = torch.stack([P.split_filter_reduce(m, c.t, c.y, c.mask, c.R, tp, tn, c.ws, smoother=False)
                        for c, (tp, tn) in zip(chunks, ends)])
    for r, c in enumerate(chunks):
        _, _, llr = P.split_filter_finish(m, c.t, c.y, c.mask, c.R, ends[r][1], aggs, r, c.ws, smoother=False,
                                          outputs=False)
        assert P.status(c.ws) == 0
        tot += float(llr.item())
    assert abs(tot - float(ll.item())) <= 1e-11 * max(abs(float(ll.item())), t.size)
    assert abs(lls - float(ll.item())) <= 1e-11 * max(abs(float(ll.item())), t.size)


def test_split_full_size_rbf(report):
    """The 2^20 + 10^4 workload (RBF-6) in 4 chunks: the posterior at the
    prediction times against the unsplit pssgp_predict and, at every 97th
    prediction time and in total, against the oracle."""
    s = wl.sinusoid_large()
    t, y, mask, tpos = oracle.merge(s.t_train, s.y_train, s.t_test)
    m = P.build_model("rbf", 1.0, 1.0)
    fm, fv, ll, _ = run_split(m, t, y, mask, 0.01, split.chunk_bounds(t.size, 4))
    mean, var, ll1, ws = P.predict(m, dev(s.t_train), dev(s.y_train), dev(s.t_test), 0.01)
    assert P.status(ws) == 0
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    em = np.max(np.abs(fm[tpos] - mean) / np.maximum(np.abs(mean), np.sqrt(var)))
    ev = np.max(np.abs(fv[tpos] - var) / var)
    report("split 2^20 rbf vs unsplit pssgp_predict (mean, variance)", max(em, ev), 1e-9)
    assert em <= 1e-9 and ev <= 1e-9
    assert abs(ll - float(ll1.item())) <= 1e-11 * max(abs(ll), s.N)
    res = oracle.run(om.make_model("rbf", 1.0, 1.0), t, y, mask, 0.01)
    pick = tpos[::97]
    check(fm[pick], fv[pick], ll, res.f_mean[pick], res.f_var[pick], res.loglik, s.N, 1e-6, report, "2^20 rbf")
