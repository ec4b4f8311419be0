"""GPU parity of the learned initialisation's pieces against the oracle, and
an end-to-end check of what the trained network gains.

* Prior simulation: the same Philox4x32-10 draws on both sides; the oracle
  builds each series' model at its own hyperparameters in its own (unbalanced)
  coordinates, the device rescales one balanced unit model; the Cholesky
  factor is covariant under the positive diagonal change of coordinates, so
  y agrees up to rounding.
* Features: FP32 sums on the device (phase re-anchored every 128 steps) against
  float64 direct sums; |d log P_j| <= 2e-3 (FP32 rotation error over 128 steps
  relative to the sums), |d log s2| <= 1e-6 (features are stored in FP32).
* Network: the oracle rounds to bfloat16 at the same points in float64; the
  device accumulates in FP32, so a value within the FP32/FP64 difference of a
  bfloat16 rounding boundary may round the other way (one bfloat16 unit,
  2^-8 relative).  Outputs: max |d| <= 2^-6 max(1, |out|max).  Gradient,
  entry by entry within each parameter block (weights, biases of each layer),
  with s = |ref| + rms(ref over the block): every entry |d| <= 1e-2 s, and at
  most 1 % of the block's entries above 1e-3 s.  A flipped rounding of one
  activation moves one of the batch's 512 terms of a weight-gradient entry by
  2^-8 of itself, far below 1e-3 s; a layout or index mistake (a transposed
  tile, a wrong row) moves whole rows or columns by O(s).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2102_09964_b300 as P
import workloads as wl
from oracle import features as of
from oracle import mlp as omlp
from oracle import model as om

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("kind", ["matern32", "matern52"])
def test_simulation_matches_oracle(kind):
    offsets, params = wl.prior_spec(61, 40, n_min=1, n_max=3000)
    m = P.build_model(kind, 1.0, 1.0)
    t, y, st = P.simulate_prior(m, dev(offsets, torch.int64), dev(params), seed=12345)
    assert int(st.item()) == 0
    t, y = t.cpu().numpy(), y.cpu().numpy()
    for s in (0, 1, 7, 20, 39):
        a, b = offsets[s], offsets[s + 1]
        mo = om.make_model(kind, params[s, 0], params[s, 1])
        rt, ry = oracle.simulate_series(mo, params[s, 2], b - a, 12345, s)
        assert np.all(np.abs(t[a:b] - rt) <= 1e-12 * (1.0 + rt)), s
        sd = math.sqrt(params[s, 1] + params[s, 2])
        assert np.all(np.abs(y[a:b] - ry) <= 1e-9 * (sd + np.abs(ry))), (s, np.max(np.abs(y[a:b] - ry)))


def test_features_match_oracle():
    offsets, params = wl.prior_spec(62, 24, n_min=2, n_max=20_000)
    offsets[3] = offsets[2]                     # an empty series (offsets stay non-decreasing)
    rng = np.random.default_rng(63)
    n = int(offsets[-1])
    t = np.empty(n)
    y = np.empty(n)
    for s in range(24):
        a, b = offsets[s], offsets[s + 1]
        t[a:b] = np.cumsum(rng.exponential(0.01, b - a))
        w = rng.uniform(0.5, 50.0)
        y[a:b] = np.sin(w * t[a:b]) + rng.normal(0, 0.3, b - a)
    y[offsets[5]:offsets[6]] = 1.5              # a constant series
    f = P.features(dev(offsets, torch.int64), dev(t), dev(y)).cpu().numpy()
    for s in range(24):
        a, b = offsets[s], offsets[s + 1]
        ref = of.features(t[a:b], y[a:b]).astype(np.float64) if b > a else np.zeros(65)
        assert np.max(np.abs(f[s, :64] - ref[:64])) <= 2e-3, (s, np.max(np.abs(f[s, :64] - ref[:64])))
        assert abs(f[s, 64] - ref[64]) <= 1e-6 * max(1.0, abs(ref[64])), s


def test_network_outputs_and_gradient_match_oracle(report):
    rng = np.random.default_rng(64)
    M = 512
    feat = rng.normal(size=(M, 65)).astype(np.float32)
    theta = rng.normal(size=(M, 3))
    norm = np.zeros(144)
    norm[:65] = rng.normal(0, 0.1, 65)
    norm[65:130] = rng.uniform(0.5, 2.0, 65)
    norm[130:133] = rng.normal(0, 0.2, 3)
    norm[133:136] = rng.uniform(0.5, 2.0, 3)
    norm = norm.astype(np.float32).astype(np.float64)
    p = omlp.random_params(65)
    net = P.MLP()
    net.set_params(p, norm)
    out = torch.full((M, 16), float("nan"), dtype=torch.float32, device="cuda")
    g, loss = net.grad(dev(feat, torch.float32), dev(theta), out=out)
    g, loss, out = g.cpu().numpy().astype(np.float64), float(loss.item()), out.cpu().numpy()
    rloss, rg, rout = omlp.loss_grad(p, norm, feat, theta)
    assert np.max(np.abs(out - rout)) <= 2.0 ** -6 * max(1.0, np.max(np.abs(rout)))
    assert abs(loss - rloss) <= 1e-2 * rloss
    blocks = [(omlp.OW1, omlp.OB1), (omlp.OB1, omlp.OW2), (omlp.OW2, omlp.OB2), (omlp.OB2, omlp.OW3),
              (omlp.OW3, omlp.OB3), (omlp.OB3, omlp.NP)]
    for a, b in blocks:
        d = np.abs(g[a:b] - rg[a:b])
        sc = np.abs(rg[a:b]) + np.sqrt(np.mean(rg[a:b] ** 2)) + 1e-30
        worst = float(np.max(d / sc))
        frac = float(np.mean(d > 1e-3 * sc))
        report(f"MLP gradient entrywise |d|/(|ref|+rms), block {a}:{b}", worst, 1e-2)
        report(f"MLP gradient fraction of entries above 1e-3, block {a}:{b}", frac, 1e-2)
        assert worst <= 1e-2, (a, b, worst, int(np.argmax(d / sc)))
        assert frac <= 1e-2, (a, b, frac)
    # padding stays exactly zero
    assert np.all(g[omlp.OW1:omlp.OB1].reshape(256, 80)[:, 65:] == 0.0)
    assert np.all(g[omlp.OW3:omlp.OB3].reshape(16, 256)[3:] == 0.0)


def _prior_data(seed, B, n=None, n_min=None, n_max=None, sim_seed=7):
    offsets, params = wl.prior_spec(seed, B, n=n, n_min=n_min, n_max=n_max)
    m = P.build_model("matern52", 1.0, 1.0)
    off = dev(offsets, torch.int64)
    t, y, st = P.simulate_prior(m, off, dev(params), seed=sim_seed)
    assert int(st.item()) == 0
    return offsets, params, off, t, y


def test_training_reduces_loss_and_predicts_hyperparameters():
    offsets, params, off, t, y = _prior_data(66, 32_768, n=1024)
    feat = P.features(off, t, y)
    theta = dev(np.log(params))
    net = P.MLP()
    net.init(3, feat, theta)
    losses = net.train(feat, theta, epochs=6, batch=2048, lr=2e-3, lr_final=2e-4).cpu().numpy()
    assert np.all(np.isfinite(losses))
    assert losses[-16:].mean() < 0.5 * losses[:4].mean()
    # held-out series: the proposals beat the constant (prior mean) guess
    offsets2, params2, off2, t2, y2 = _prior_data(67, 1024, n=1024, sim_seed=8)
    pred = net.predict(P.features(off2, t2, y2)).cpu().numpy()
    err = np.sqrt(np.mean((pred - np.log(params2)) ** 2, axis=0))
    base = np.sqrt(np.mean((np.log(params2) - np.log(params2).mean(axis=0)) ** 2, axis=0))
    assert np.all(err < 0.8 * base), (err, base)


def test_learned_init_fits_match_plain_fits_in_fewer_iterations():
    offsets, params, off, t, y = _prior_data(68, 65_536, n=1024)
    net = P.MLP()
    net.init(4, P.features(off, t, y), dev(np.log(params)))
    net.train(P.features(off, t, y), dev(np.log(params)), epochs=6, batch=2048, lr=2e-3, lr_final=2e-4)
    ho, hp, hoff, ht, hy = _prior_data(69, 48, n_min=2048, n_max=8192, sim_seed=9)
    m = P.build_model("matern52", 1.0, 1.0)
    mask = torch.ones(ht.numel(), dtype=torch.uint8, device="cuda")
    th_plain, ll_plain, it_plain, _ = P.fit_batched(m, ho, ht, hy, mask, np.zeros((48, 3)))
    init = net.predict(P.features(hoff, ht, hy))
    th_l, ll_l, it_l, _ = P.fit_batched(m, ho, ht, hy, mask, init)
    n = np.diff(ho)
    ok = ll_l.cpu().numpy() >= ll_plain.cpu().numpy() - 1e-3 * n
    assert ok.mean() >= 0.95
    assert it_l.sum().item() < it_plain.sum().item()


def test_network_falls_back_to_the_default_init():
    """A proposal from a non-finite input (which the ReLU would otherwise
    hide), or one far outside the training targets, is replaced by the plain
    default 0 (l = s2 = R = 1)."""
    rng = np.random.default_rng(70)
    norm = np.zeros(144)
    norm[65:130] = 1.0
    norm[133:136] = 1.0
    p = omlp.random_params(71)
    net = P.MLP()
    net.set_params(p, norm)
    feat = rng.normal(size=(8, 65)).astype(np.float32)
    feat[2, 10] = np.nan
    th = net.predict(dev(feat, torch.float32)).cpu().numpy()
    out, _ = omlp.forward(p, norm, feat)
    for r in range(8):
        z = out[r, :3]
        if np.all(np.isfinite(z)) and np.any(np.abs(np.abs(z) - 4.0) < 0.05):
            continue                          # too close to the cut to compare FP32 with FP64
        ok = np.all(np.isfinite(z)) and np.all(np.abs(z) <= 4.0)
        if ok:
            assert np.allclose(th[r], z, atol=2.0 ** -6 * max(1.0, np.abs(z).max()))
        else:
            assert np.all(th[r] == 0.0)
    assert np.all(th[2] == 0.0)
