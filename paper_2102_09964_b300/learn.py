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


def compare_fits(net, model, offsets: np.ndarray, t, y, order: str = "abba", **fit_kw):
    """Plain-init and learned-init fits of the same series with the same
    options (fit_kw: options of fit_batched).  Each fit runs in the order
    given (default plain, learned, learned, plain, so that neither start
    always runs first); a fit's time is device wall clock around it (the
    learned one includes its features and the network's forward pass), and
    the mean over its runs is reported.  Returns a dict of results."""
    B = offsets.size - 1
    dev = t.device
    mask = torch.ones(t.numel(), dtype=torch.uint8, device=dev)
    off = torch.as_tensor(offsets, dtype=torch.int64, device=dev)
    runs = {"plain": [], "learned": []}
    out = {}
    for which in {"ab": ("plain", "learned"), "ba": ("learned", "plain"),
                  "abba": ("plain", "learned", "learned", "plain")}[order]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        init = np.zeros((B, 3)) if which == "plain" else net.predict(features(off, t, y))
        th, ll, it, nloop = fit_batched(model, offsets, t, y, mask, init, **fit_kw)
        torch.cuda.synchronize()
        runs[which].append(time.perf_counter() - t0)
        out[which] = (ll.cpu().numpy(), int(it.sum().item()), nloop, init)
    n = np.diff(offsets).astype(np.float64)
    (llp, itp, np_, _), (lll, itl, nl, init) = out["plain"], out["learned"]
    res = {"series": B, "steps_total": int(offsets[-1]), "order": order}
    for which, (it_total, nloop) in (("plain", (itp, np_)), ("learned", (itl, nl))):
        gs = float(np.mean(runs[which]))
        res[which] = {"gpu_s": gs, "gpu_s_runs": [round(x, 4) for x in runs[which]], "series_per_s": B / gs,
                      "iterations_total": it_total, "loop_iterations": nloop}
    res.update({
        "learned_within_1e-3_nats_per_point": float(np.mean(lll >= llp - 1e-3 * n)),
        "learned_better_by_1e-3_nats_per_point": float(np.mean(lll > llp + 1e-3 * n)),
        "theta_learned_init": init.cpu().numpy() if torch.is_tensor(init) else init,
        "loglik_plain": llp,
        "loglik_learned": lll,
    })
    return res


def heldout_series(model, offsets: np.ndarray, params: np.ndarray, seed: int, device="cuda"):
    """Device (t, y) of held-out prior series."""
    off = torch.as_tensor(offsets, dtype=torch.int64, device=device)
    par = torch.as_tensor(params, dtype=torch.float64, device=device)
    t, y, st = simulate_prior(model, off, par, seed=seed)
    return t, y
