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
    # log-likelihood only (no per-step outputs, no smoother): the per-chunk closed form (each
    # chunk's terms given the state 0 before it, corrected by the Gaussian integral over that state)
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


# ---------------------------------------------------------------------------
# the gradient over a split series (grad_protocol: the forward exchange, then
# the mean- and covariance-adjoint exchanges), against the oracle's
# forward-mode gradient of the whole series.  Tolerance as the unsplit
# gradient's: per component |g - ref| / max(|ref|, s / sqrt(n_obs),
# 1e-5 sqrt(n_obs)) <= 1e-8 (Matern), 1e-6 (RBF-6), s the oracle's sum of
# |per-step term|.
# ---------------------------------------------------------------------------
GTOL = {"matern12": 1e-8, "matern32": 1e-8, "matern52": 1e-8, "rbf": 1e-6}


def run_split_grad(m, t, y, mask, R, bounds):
    G = len(bounds)
    Rs = [R if np.isscalar(R) else dev(R[a:b]) for a, b in bounds]
    chunks = [split.LibraryChunk(m, dev(t[a:b]), dev(y[a:b]), dev(mask[a:b], torch.uint8), Rs[r], grad=True)
              for r, (a, b) in enumerate(bounds)]
    res = split.run_lockstep([split.grad_protocol(c, r, G) for r, c in enumerate(chunks)])
    for c in chunks:
        assert P.status(c.ws) == 0
    lls = {float(r[0].item()) for r in res}
    gs = {tuple(r[1].cpu().numpy().tolist()) for r in res}
    assert len(lls) == 1 and len(gs) == 1          # every rank holds the same totals
    return lls.pop(), np.array(gs.pop())


def check_split_grad(kind, ell, s2, t, y, mask, R, ll, g, report, what):
    rll, rg, sc = oracle.loglik_grad_fwd(kind, ell, s2, t, y, mask, R, with_scale=True)
    nobs = max(int(mask.sum()), 1)
    floor = np.maximum(np.asarray(sc) / np.sqrt(nobs), 1e-5 * np.sqrt(nobs))
    eg = np.max(np.abs(g - rg) / np.maximum(np.abs(rg), floor))
    el = abs(ll - rll) / max(abs(rll), nobs)
    tol = GTOL[kind]
    report(f"split gradient vs forward mode, {what} (tol {tol:g})", eg, tol)
    assert np.isfinite(eg) and eg <= tol, (what, g, rg, eg)
    assert el <= TOL.get(kind, 1e-9), (what, ll, rll)


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "rbf"])
@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_split_gradient_equals_forward_mode(kind, G, report):
    s = wl.random_series(111, 12_000, 0, T=130.0)
    rng = np.random.default_rng(112)
    mask = (rng.uniform(size=s.N) > 0.1).astype(np.uint8)
    m = P.build_model(kind, 0.7, 1.3)
    ll, g = run_split_grad(m, s.t_train, s.y_train, mask, 0.02, split.chunk_bounds(s.N, G))
    check_split_grad(kind, 0.7, 1.3, s.t_train, s.y_train, mask, 0.02, ll, g, report, f"{kind}, G={G}")


def test_split_gradient_g1_equals_the_unsplit_call():
    """One chunk runs the unsplit gradient's kernels on the same elements: the
    same sums to the last bits (a few ulps of the reduction order at most)."""
    s = wl.random_series(113, 20_000, 0, T=200.0)
    mask = np.ones(s.N, np.uint8)
    m = P.build_model("matern52", 0.9, 1.1)
    ll1, g1, ws = P.loglik_grad(m, dev(s.t_train), dev(s.y_train), dev(mask, torch.uint8), 0.03)
    assert P.status(ws) == 0
    ll, g = run_split_grad(m, s.t_train, s.y_train, mask, 0.03, [(0, s.N)])
    g1 = g1.cpu().numpy()
    assert abs(ll - float(ll1.item())) <= 1e-13 * abs(ll)
    assert np.all(np.abs(g - g1) <= 1e-12 * np.maximum(np.abs(g1), 1.0))


def test_split_gradient_uneven_chunks_gaps_ties_and_per_step_noise(report):
    """Chunks of 1, 2 and 33 steps, a chunk that is one missing step, a chunk
    boundary across a gap of 40 lengthscales and one inside a run of ties
    (a zero-length transition between chunks), per-step noise variances."""
    s = wl.random_series(114, 6_000, 0, T=66.0)
    t = s.t_train.copy()
    t[3300:] += 40.0
    t[4999:5003] = t[4999]
    mask = (np.random.default_rng(115).uniform(size=s.N) > 0.2).astype(np.uint8)
    mask[3300] = 0
    mask[36] = 0
    R = np.exp(np.random.default_rng(116).uniform(np.log(1e-3), np.log(1e-1), s.N))
    bounds = [(0, 1), (1, 3), (3, 36), (36, 37), (37, 3300), (3300, 5001), (5001, s.N)]
    for kind in ("matern32", "rbf"):
        m = P.build_model(kind, 1.0, 1.0)
        ll, g = run_split_grad(m, t, s.y_train, mask, R, bounds)
        check_split_grad(kind, 1.0, 1.0, t, s.y_train, mask, R, ll, g, report, f"uneven chunks, {kind}")


def test_split_gradient_full_size_rbf(report):
    """2^20 training steps (RBF-6) in 4 chunks against the unsplit library
    gradient and the oracle's forward mode."""
    s = wl.sinusoid_large(M=0)
    mask = np.ones(s.N, np.uint8)
    m = P.build_model("rbf", 1.0, 1.0)
    ll, g = run_split_grad(m, s.t_train, s.y_train, mask, 0.01, split.chunk_bounds(s.N, 4))
    ll1, g1, ws = P.loglik_grad(m, dev(s.t_train), dev(s.y_train), dev(mask, torch.uint8), 0.01)
    assert P.status(ws) == 0
    g1 = g1.cpu().numpy()
    e1 = np.max(np.abs(g - g1) / np.maximum(np.abs(g1), 1e-5 * np.sqrt(s.N)))
    report("split 2^20 rbf gradient vs unsplit pssgp_loglik_grad", e1, 1e-8)
    assert e1 <= 1e-8 and abs(ll - float(ll1.item())) <= 1e-11 * max(abs(ll), s.N)
    check_split_grad("rbf", 1.0, 1.0, s.t_train, s.y_train, mask, 0.01, ll, g, report, "2^20 rbf")
