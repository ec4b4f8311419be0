"""One long series split in contiguous time chunks over G ranks, one GPU each.

The filter and the smoother are scans of associative operators (Sec. 3 and
Prop. 1; supplement Prop. 2), so a series cut into G chunks needs one
exchange per direction: each rank reduces its chunk to one filter aggregate,
the ranks all-gather the G aggregates, each rank folds those before it into
the state its chunk starts from and filters its chunk; the smoother does the
same backwards with the aggregates after it.  The log-likelihood is the sum
of the chunks' terms (each given all earlier data), one all-reduce.

The gradient of the log-likelihood by the adjoint scans splits the same way:
the forward exchange as above, then one backward exchange for the adjoint of
the predicted means and one for that of the predicted covariances (both of
the smoothing operator's form), and an all-reduce of the chunks' terms.

The rank's side of the exchange is written once, as a generator
(``chunk_protocol``) that yields every collective it needs:
``("all_gather", tensor)`` is answered with the [G, ...] stack of every
rank's tensor in rank order, ``("all_reduce_sum", tensor)`` with the sum.
``run_distributed`` answers them with torch.distributed (one process per
GPU; NCCL, or gloo on CPU), ``run_lockstep`` steps the generators of all
ranks together in one process (several chunks on one device: nothing waits
on the GPU for anything but its own earlier work).  The chunk's arithmetic
is the backend's; ``LibraryChunk`` runs every step in libpssgp's kernels
through the C ABI (pssgp_split_*).
"""
from __future__ import annotations

import math

import torch

from . import (Model, split_filter_finish, split_filter_reduce, split_grad_finish, split_grad_mean_finish,
               split_grad_mean_reduce, split_smooth_finish, split_smooth_reduce, workspace, workspace_grad)


def chunk_protocol(chunk, rank: int, G: int):
    """Rank `rank` of G: yields collectives, returns (f_mean, f_var, loglik)
    of its chunk (loglik: the whole series', the same on every rank)."""
    ends = yield ("all_gather", chunk.time_ends())          # [G, 2]: first and last time of each chunk
    t_prev = float(ends[rank - 1, 1]) if rank > 0 else math.nan
    t_next = float(ends[rank + 1, 0]) if rank + 1 < G else math.nan
    aggs_f = yield ("all_gather", chunk.filter_reduce(t_prev, t_next))
    ll = chunk.filter_finish(aggs_f, rank)
    aggs_s = yield ("all_gather", chunk.smooth_reduce())
    ll_total = yield ("all_reduce_sum", ll)
    f_mean, f_var = chunk.smooth_finish(aggs_s, rank)
    return f_mean, f_var, ll_total


def grad_protocol(chunk, rank: int, G: int):
    """Rank `rank` of G: yields collectives, returns (loglik, grad[3]) of the
    whole series (the same on every rank)."""
    ends = yield ("all_gather", chunk.time_ends())
    t_prev = float(ends[rank - 1, 1]) if rank > 0 else math.nan
    t_next = float(ends[rank + 1, 0]) if rank + 1 < G else math.nan
    aggs_f = yield ("all_gather", chunk.filter_reduce(t_prev, t_next))
    ll = chunk.filter_finish(aggs_f, rank)
    aggs_m = yield ("all_gather", chunk.mean_adjoint_reduce())
    aggs_c = yield ("all_gather", chunk.mean_adjoint_finish(aggs_m, rank))
    g = chunk.grad_finish(aggs_c, rank)
    tot = yield ("all_reduce_sum", torch.cat([ll.reshape(1), g.reshape(3)]))
    return tot[0], tot[1:]


def run_distributed(gen, group=None):
    """Drive one rank's protocol with torch.distributed collectives."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    msg = None
    while True:
        try:
            kind, x = gen.send(msg)
        except StopIteration as stop:
            return stop.value
        x = x.contiguous()
        if kind == "all_gather":
            parts = [torch.empty_like(x) for _ in range(world)]
            dist.all_gather(parts, x, group=group)
            msg = torch.stack(parts)
        elif kind == "all_reduce_sum":
            msg = x.clone()
            dist.all_reduce(msg, group=group)
        else:
            raise ValueError(f"unknown collective {kind!r}")


def run_lockstep(gens):
    """Drive the protocols of all G ranks in one process, answering each
    collective once every rank has reached it; returns every rank's result."""
    G = len(gens)
    msgs = [None] * G
    results = [None] * G
    done = [False] * G
    while not all(done):
        reqs = {}
        for r in range(G):
            if done[r]:
                continue
            try:
                reqs[r] = gens[r].send(msgs[r])
            except StopIteration as stop:
                results[r] = stop.value
                done[r] = True
        if not reqs:
            break
        if len(reqs) != G:
            raise RuntimeError("the ranks left the exchange at different points")
        kinds = {k for k, _ in reqs.values()}
        if len(kinds) != 1:
            raise RuntimeError(f"the ranks asked for different collectives: {sorted(kinds)}")
        kind = kinds.pop()
        xs = [reqs[r][1] for r in range(G)]
        if kind == "all_gather":
            out = torch.stack(xs)
            msgs = [out] * G
        elif kind == "all_reduce_sum":
            out = xs[0].clone()
            for x in xs[1:]:
                out += x
            msgs = [out.clone() for _ in range(G)]
        else:
            raise ValueError(f"unknown collective {kind!r}")
    return results


class LibraryChunk:
    """One rank's chunk on its GPU: sorted times t, observations y, mask (1
    observed, 0 missing), noise variance R (scalar or per step); device
    tensors.  The workspace carries each call's state to the next.  The
    filter pass also forms the smoother elements (fused, as in the prediction
    path); with `filter_outputs` it writes the filter states too.  With
    `grad` the chunk runs grad_protocol (the adjoint passes) instead."""

    def __init__(self, model: Model, t, y, mask, R, ws=None, filter_outputs=False, grad=False):
        self.model, self.t, self.y, self.mask, self.R = model, t, y, mask, R
        self.grad = grad
        if ws is None:
            ws = (workspace_grad if grad else workspace)(model.d, t.numel(), t.device)
        self.ws = ws
        self.filter_outputs = filter_outputs
        self.xf = self.Pf = None
        self.t_next = math.nan

    def time_ends(self):
        return torch.stack([self.t[0], self.t[-1]])

    def filter_reduce(self, t_prev: float, t_next: float):
        self.t_next = t_next
        return split_filter_reduce(self.model, self.t, self.y, self.mask, self.R, t_prev, t_next, self.ws,
                                   grad=self.grad)

    def filter_finish(self, aggs, rank: int):
        self.xf, self.Pf, ll = split_filter_finish(self.model, self.t, self.y, self.mask, self.R, self.t_next, aggs,
                                                   rank, self.ws, outputs=self.filter_outputs, grad=self.grad)
        return ll

    def mean_adjoint_reduce(self):
        return split_grad_mean_reduce(self.model, self.t.numel(), self.ws, device=self.t.device)

    def mean_adjoint_finish(self, aggs, rank: int):
        return split_grad_mean_finish(self.model, self.t.numel(), aggs, rank, self.ws, device=self.t.device)

    def grad_finish(self, aggs, rank: int):
        return split_grad_finish(self.model, self.t.numel(), self.R, aggs, rank, self.ws, device=self.t.device)

    def smooth_reduce(self):
        return split_smooth_reduce(self.model, self.t.numel(), self.ws, device=self.t.device)

    def smooth_finish(self, aggs, rank: int):
        fm, fv, _, _ = split_smooth_finish(self.model, self.t.numel(), aggs, rank, self.ws, device=self.t.device)
        return fm, fv


def chunk_bounds(n: int, G: int):
    """Contiguous chunks of n steps for G ranks, as equal as possible."""
    if G < 1 or n < G:
        raise ValueError("need at least one step per rank")
    return [(r * n // G, (r + 1) * n // G) for r in range(G)]


def split_filter_smoother(model: Model, t, y, mask, R: float, G: int):
    """The whole series cut into G chunks, all ranks run in lockstep in this
    process (one device): returns (f_mean, f_var, loglik) over all steps."""
    chunks = [LibraryChunk(model, t[a:b], y[a:b], mask[a:b], R) for a, b in chunk_bounds(t.numel(), G)]
    res = run_lockstep([chunk_protocol(c, r, G) for r, c in enumerate(chunks)])
    return torch.cat([r[0] for r in res]), torch.cat([r[1] for r in res]), res[0][2]


def split_loglik_grad(model: Model, t, y, mask, R, G: int):
    """The log-likelihood of the whole series and its gradient (as
    loglik_grad) with the series cut into G chunks, all ranks run in lockstep
    in this process (one device): returns (loglik, grad[3]) as device tensors."""
    chunks = [LibraryChunk(model, t[a:b], y[a:b], mask[a:b], R if _scalar(R) else R[a:b], grad=True)
              for a, b in chunk_bounds(t.numel(), G)]
    res = run_lockstep([grad_protocol(c, r, G) for r, c in enumerate(chunks)])
    return res[0]


def _scalar(R) -> bool:
    return not torch.is_tensor(R) or R.numel() == 1
