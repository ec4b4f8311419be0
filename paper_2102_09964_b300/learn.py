"""The learned initialisation of the batched marginal-likelihood fit, end to
end on the device: simulate training series from the state-space prior,
extract their features, train the network, and compare fits started from its
proposals with fits started from the plain default (l = s2 = R = 1).

Every step runs in the library's kernels; this module only sequences the
calls and moves the small per-series tables.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import MLP, NFEAT, _empty, features, fit_batched, simulate_prior


def prior_features(model, offsets: np.ndarray, params: np.ndarray, seed: int, chunk: int = 65_536,
                   device="cuda"):
    """Features (device float32[B, 65]) of B series drawn from the model's
    prior, simulated `chunk` series at a time (chunk c uses key seed + c, so
    the chunks draw independent numbers); the series themselves are not kept."""
    B = offsets.size - 1
    feat = _empty(B, NFEAT, dtype=torch.float32, device=device)
    for c, a in enumerate(range(0, B, chunk)):
        b = min(a + chunk, B)
        off = torch.as_tensor(offsets[a:b + 1] - offsets[a], dtype=torch.int64, device=device)
        par = torch.as_tensor(params[a:b], dtype=torch.float64, device=device)
        t, y, st = simulate_prior(model, off, par, seed=seed + c)
        features(off, t, y, out=feat[a:b])
        del t, y
    return feat


def train_network(model, offsets, params, seed: int, epochs: int = 8, batch: int = 4096, lr: float = 2e-3,
                  lr_final: float = 1e-4, device="cuda"):
    """Simulate, featurise and train; returns (network, seconds, losses)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    feat = prior_features(model, offsets, params, seed, device=device)
    theta = torch.as_tensor(np.log(params), dtype=torch.float64, device=device)
    net = MLP(device)
    net.init(seed, feat, theta)
    losses = net.train(feat, theta, epochs=epochs, batch=batch, lr=lr, lr_final=lr_final)
    torch.cuda.synchronize()
    return net, time.perf_counter() - t0, losses


def compare_fits(net, model, offsets: np.ndarray, t, y, **fit_kw):
    """Plain-init and learned-init fits of the same series.  Times are device
    wall-clock around each fit (the learned one includes its features and
    the network's forward pass).  fit_kw: options of fit_batched (the same
    for both fits).  Returns a dict of results."""
    B = offsets.size - 1
    dev = t.device
    mask = torch.ones(t.numel(), dtype=torch.uint8, device=dev)
    off = torch.as_tensor(offsets, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th_p, ll_p, it_p, n_p = fit_batched(model, offsets, t, y, mask, np.zeros((B, 3)), **fit_kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    init = net.predict(features(off, t, y))
    th_l, ll_l, it_l, n_l = fit_batched(model, offsets, t, y, mask, init, **fit_kw)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n = np.diff(offsets).astype(np.float64)
    llp, lll = ll_p.cpu().numpy(), ll_l.cpu().numpy()
    return {
        "series": B,
        "steps_total": int(offsets[-1]),
        "plain": {"gpu_s": t1 - t0, "series_per_s": B / (t1 - t0), "iterations_total": int(it_p.sum().item()),
                  "loop_iterations": n_p},
        "learned": {"gpu_s": t2 - t1, "series_per_s": B / (t2 - t1), "iterations_total": int(it_l.sum().item()),
                    "loop_iterations": n_l},
        "learned_within_1e-3_nats_per_point": float(np.mean(lll >= llp - 1e-3 * n)),
        "learned_better_by_1e-3_nats_per_point": float(np.mean(lll > llp + 1e-3 * n)),
        "theta_learned_init": init.cpu().numpy(),
        "loglik_plain": llp,
        "loglik_learned": lll,
    }


def heldout_series(model, offsets: np.ndarray, params: np.ndarray, seed: int, device="cuda"):
    """Device (t, y) of held-out prior series."""
    off = torch.as_tensor(offsets, dtype=torch.int64, device=device)
    par = torch.as_tensor(params, dtype=torch.float64, device=device)
    t, y, st = simulate_prior(model, off, par, seed=seed)
    return t, y
