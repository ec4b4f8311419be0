"""One long series split in time chunks over several ranks: the exchange of
paper_2102_09964_b300.split (which aggregates each rank folds, in which
order, the neighbours' boundary times) checked on CPU ranks with the
oracle's arithmetic.

The chunk backend here (test infrastructure) computes each step of a rank
with the oracle: the filtering and smoothing elements and operators of Sec. 3
and supplement Prop. 2 (folded sequentially), and the sequential filter from
a start state (``kalman_filter_from``).  The exchange runs on 2 and 3
``gloo`` processes and in lockstep in one process; the concatenated result
must equal the single-rank oracle (sequential Kalman filter and RTS smoother
over the whole series) at the tolerances of the GPU parity tests.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as wl
from oracle import model as om
from paper_2102_09964_b300 import split

TOL = {"matern32": 1e-9, "matern52": 1e-9, "rbf": 1e-6}


def _pack(parts):
    return torch.as_tensor(np.concatenate([np.ravel(p) for p in parts]), dtype=torch.float64)


def _unpack(v, d, sizes):
    v = np.asarray(v, dtype=np.float64)
    out, o = [], 0
    for shape in sizes(d):
        k = int(np.prod(shape))
        out.append(v[o:o + k].reshape(shape))
        o += k
    return tuple(out)


def _fsizes(d):
    return [(d, d), (d,), (d, d), (d,), (d, d)]


def _ssizes(d):
    return [(d, d), (d,), (d, d)]


class OracleChunk:
    """One rank's chunk, every step by the oracle (CPU, float64 tensors)."""

    def __init__(self, m, t, y, mask, R):
        self.m, self.t, self.y, self.mask, self.R = m, t, y, mask, R
        self.d = m.d

    def time_ends(self):
        return torch.tensor([self.t[0], self.t[-1]], dtype=torch.float64)

    def filter_reduce(self, t_prev, t_next):
        m, n = self.m, self.t.size
        self.t_next = t_next
        if math.isnan(t_prev):
            self.F, self.Q = oracle.discretize(m, self.t)
            el = oracle.filter_elements(m, self.F, self.Q, self.y, self.mask, self.R)
            el = [x for x in el]
        else:
            # a leading masked step at t_prev: the elements after it are the
            # chunk's, with the transition from t_prev into step 0
            tt = np.concatenate([[t_prev], self.t])
            F, Q = oracle.discretize(m, tt)
            self.F, self.Q = F[1:], Q[1:]
            el = oracle.filter_elements(m, F, Q, np.concatenate([[0.0], self.y]),
                                        np.concatenate([[0], self.mask]).astype(np.uint8), self.R)
            el = [x[1:] for x in el]
        acc = tuple(x[0] for x in el)
        for k in range(1, n):
            acc = oracle.filter_combine(acc, tuple(x[k] for x in el))
        return _pack(acc)

    def filter_finish(self, aggs, rank):
        m = self.m
        if rank == 0:
            self.mo, self.Po, _, _, ll = oracle.kalman_filter(m, self.F, self.Q, self.y, self.mask, self.R)
        else:
            acc = _unpack(aggs[0], self.d, _fsizes)
            for r in range(1, rank):
                acc = oracle.filter_combine(acc, _unpack(aggs[r], self.d, _fsizes))
            self.mo, self.Po, _, _, ll = oracle.kalman_filter_from(m, acc[1], acc[2], self.F, self.Q, self.y,
                                                                   self.mask, self.R)
        return torch.tensor([ll], dtype=torch.float64)

    def smooth_reduce(self):
        m, n, t_next = self.m, self.t.size, self.t_next
        if math.isnan(t_next):
            self.el = oracle.smoother_elements(self.F, self.Q, self.mo, self.Po)
        else:
            # a trailing step at t_next: element n-1 is the transition into it
            F, Q = oracle.discretize(m, np.concatenate([self.t[-1:], [t_next]]))
            Fx = np.concatenate([self.F, F[1:]])
            Qx = np.concatenate([self.Q, Q[1:]])
            el = oracle.smoother_elements(Fx, Qx, np.concatenate([self.mo, self.mo[-1:]]),
                                          np.concatenate([self.Po, self.Po[-1:]]))
            self.el = [x[:n] for x in el]
        acc = tuple(x[n - 1] for x in self.el)
        for k in range(n - 2, -1, -1):
            acc = oracle.smoother_combine(tuple(x[k] for x in self.el), acc)
        return _pack(acc)

    def smooth_finish(self, aggs, rank):
        n, G = self.t.size, aggs.shape[0]
        acc = None
        for r in range(G - 1, rank, -1):
            e = _unpack(aggs[r], self.d, _ssizes)
            acc = e if acc is None else oracle.smoother_combine(e, acc)
        H = self.m.H.ravel()
        fm, fv = np.empty(n), np.empty(n)
        for k in range(n - 1, -1, -1):
            e = tuple(x[k] for x in self.el)
            acc = e if acc is None else oracle.smoother_combine(e, acc)
            fm[k] = H @ acc[1]
            fv[k] = H @ acc[2] @ H
        return torch.as_tensor(fm), torch.as_tensor(fv)


def _series(kind, n_train=1500, n_test=150, seed=91):
    s = wl.random_series(seed, n_train, n_test, T=0.01 * (n_train + n_test))
    t, y, mask, _ = oracle.merge(s.t_train, s.y_train, s.t_test)
    m = om.make_model(kind, 0.3, 1.1)
    return m, t, y, mask


def _check(kind, m, t, y, mask, R, fm, fv, ll):
    res = oracle.run(m, t, y, mask, R)
    tol = TOL[kind]
    em = np.max(np.abs(fm - res.f_mean) / np.maximum(np.abs(res.f_mean), np.sqrt(res.f_var)))
    ev = np.max(np.abs(fv - res.f_var) / res.f_var)
    el = abs(ll - res.loglik) / max(abs(res.loglik), int(mask.sum()))
    assert em <= tol and ev <= tol and el <= tol, (em, ev, el)


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_lockstep_exchange_equals_the_single_rank_oracle(oracle_lib, kind, G):
    m, t, y, mask = _series(kind)
    bounds = split.chunk_bounds(t.size, G)
    gens = [split.chunk_protocol(OracleChunk(m, t[a:b], y[a:b], mask[a:b], 0.02), r, G)
            for r, (a, b) in enumerate(bounds)]
    res = split.run_lockstep(gens)
    fm = np.concatenate([r[0].numpy() for r in res])
    fv = np.concatenate([r[1].numpy() for r in res])
    lls = {float(r[2]) for r in res}
    assert len(lls) == 1                           # every rank holds the same total
    _check(kind, m, t, y, mask, 0.02, fm, fv, lls.pop())


def test_chunks_of_one_step_and_a_missing_boundary(oracle_lib):
    """Chunks of a single step; a rank whose chunk is one unobserved step."""
    m, t, y, mask = _series("matern52", 40, 6, seed=92)
    mask = mask.copy()
    G = 7
    bounds = [(0, 1), (1, 2), (2, 3), (3, 20), (20, 21), (21, 45), (45, 46)]
    mask[20] = 0
    gens = [split.chunk_protocol(OracleChunk(m, t[a:b], y[a:b], mask[a:b], 0.02), r, G)
            for r, (a, b) in enumerate(bounds)]
    res = split.run_lockstep(gens)
    _check("matern52", m, t, y, mask, 0.02, np.concatenate([r[0].numpy() for r in res]),
           np.concatenate([r[1].numpy() for r in res]), float(res[0][2]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        m, t, y, mask = _series(kind)
        a, b = split.chunk_bounds(t.size, world)[rank]
        fm, fv, ll = split.run_distributed(
            split.chunk_protocol(OracleChunk(m, t[a:b], y[a:b], mask[a:b], 0.02), rank, world))
        out[rank] = (fm.numpy().tolist(), fv.numpy().tolist(), float(ll))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_single_rank_oracle(oracle_lib, world):
    kind = "matern52"
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, kind, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == list(range(world))
    fm = np.concatenate([res[r][0] for r in range(world)])
    fv = np.concatenate([res[r][1] for r in range(world)])
    assert len({res[r][2] for r in range(world)}) == 1
    m, t, y, mask = _series(kind)
    _check(kind, m, t, y, mask, 0.02, fm, fv, res[0][2])


class RecordingGradChunk:
    """A chunk for grad_protocol whose every result encodes (rank, stage), and
    which checks what each exchange hands it: the [G, ...] stack of all ranks'
    results of the stage in rank order, and the neighbours' boundary times."""

    def __init__(self, rank, G, t):
        self.rank, self.G, self.t = rank, G, t
        self.seen = []

    def _mine(self, stage):
        return torch.tensor([100.0 * self.rank + stage, float(self.G)], dtype=torch.float64)

    def _check_stack(self, aggs, stage):
        want = torch.stack([torch.tensor([100.0 * r + stage, float(self.G)], dtype=torch.float64)
                            for r in range(self.G)])
        assert torch.equal(aggs, want)
        self.seen.append(stage)

    def time_ends(self):
        return torch.tensor([self.t[0], self.t[-1]], dtype=torch.float64)

    def filter_reduce(self, t_prev, t_next):
        r = self.rank
        assert math.isnan(t_prev) if r == 0 else t_prev == 10.0 * r - 1.0
        assert math.isnan(t_next) if r + 1 == self.G else t_next == 10.0 * (r + 1)
        return self._mine(1)

    def filter_finish(self, aggs, rank):
        assert rank == self.rank
        self._check_stack(aggs, 1)
        return torch.tensor([float(rank + 1)], dtype=torch.float64)

    def mean_adjoint_reduce(self):
        return self._mine(2)

    def mean_adjoint_finish(self, aggs, rank):
        self._check_stack(aggs, 2)
        return self._mine(3)

    def grad_finish(self, aggs, rank):
        self._check_stack(aggs, 3)
        return torch.tensor([1.0, float(rank), -2.0], dtype=torch.float64)


def _recording_chunks(G):
    return [RecordingGradChunk(r, G, np.array([10.0 * r, 10.0 * r + 5.0, 10.0 * r + 9.0])) for r in range(G)]


def _grad_totals(G):
    return G * (G + 1) / 2, [float(G), G * (G - 1) / 2, -2.0 * G]


@pytest.mark.parametrize("G", [1, 2, 4])
def test_grad_protocol_exchanges_in_lockstep(G):
    chunks = _recording_chunks(G)
    res = split.run_lockstep([split.grad_protocol(c, r, G) for r, c in enumerate(chunks)])
    ll, g = _grad_totals(G)
    for c, (rll, rg) in zip(chunks, res):
        assert c.seen == [1, 2, 3]
        assert float(rll) == ll and rg.tolist() == g


def _grad_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = _recording_chunks(world)[rank]
        ll, g = split.run_distributed(split.grad_protocol(c, rank, world))
        out[rank] = (c.seen, float(ll), g.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_grad_protocol_on_gloo_ranks():
    world = 3
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_grad_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    ll, g = _grad_totals(world)
    assert sorted(res) == list(range(world))
    for r in range(world):
        assert res[r] == ([1, 2, 3], ll, g)


def test_lockstep_rejects_ranks_that_disagree():
    def a():
        yield ("all_gather", torch.zeros(1))

    def b():
        yield ("all_reduce_sum", torch.zeros(1))

    with pytest.raises(RuntimeError):
        split.run_lockstep([a(), b()])
