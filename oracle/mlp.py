"""Oracle of the learned initialisation's network: forward pass, loss and
gradient of the 65 -> 256 -> 256 -> 3 ReLU network in float64, with values
rounded to bfloat16 (round to nearest, ties to even) exactly where the
device path stores bfloat16: the standardised inputs, the weights, the two
hidden activations, the loss gradient at the outputs and the two hidden
gradients.  Everything else (accumulation, biases, outputs, weight
gradients) is float64 here and float32 on the device.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Parameter layout (flat float array): W1[256][80] (columns >= 65 zero),
b1[256], W2[256][256], b2[256], W3[16][256] (rows >= 3 zero), b3[16].
Normalisation: feature mean[65], sd[65], target mean[3], sd[3].
Loss: 1/(2M) sum over the M rows and 3 outputs of (out - (theta - mu)/sd)^2.
"""
from __future__ import annotations

import numpy as np

HID, KIN, NOUT, NF = 256, 80, 16, 65
OW1 = 0
OB1 = OW1 + HID * KIN
OW2 = OB1 + HID
OB2 = OW2 + HID * HID
OW3 = OB2 + HID
OB3 = OW3 + NOUT * HID
NP = OB3 + NOUT


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return (p[OW1:OB1].reshape(HID, KIN), p[OB1:OW2], p[OW2:OB2].reshape(HID, HID), p[OB2:OW3],
            p[OW3:OB3].reshape(NOUT, HID), p[OB3:NP])


def forward(p, norm, feat, rounding=True):
    """Returns (out[M][16], cache).  rounding=False: no bfloat16 rounding
    (the plain float64 network, for the finite-difference pins)."""
    r = bf16 if rounding else (lambda x: np.asarray(x, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    norm = np.asarray(norm, dtype=np.float64)
    M = feat.shape[0]
    X = np.zeros((M, KIN))
    X[:, :NF] = (np.asarray(feat, dtype=np.float32).astype(np.float64) - norm[:NF]) / norm[NF:2 * NF]
    X = r(X)
    W1h, W2h, W3h = r(W1), r(W2), r(W3)
    H1 = r(np.maximum(X @ W1h.T + b1, 0.0))
    H2 = r(np.maximum(H1 @ W2h.T + b2, 0.0))
    out = H2 @ W3h.T + b3
    return out, (X, H1, H2, W1h, W2h, W3h)


def loss_grad(p, norm, feat, theta, rounding=True):
    """(loss, grad[NP], out) of the training loss."""
    r = bf16 if rounding else (lambda x: np.asarray(x, dtype=np.float64))
    out, (X, H1, H2, W1h, W2h, W3h) = forward(p, norm, feat, rounding)
    norm = np.asarray(norm, dtype=np.float64)
    M = feat.shape[0]
    tn = (np.asarray(theta, dtype=np.float64) - norm[2 * NF:2 * NF + 3]) / norm[2 * NF + 3:2 * NF + 6]
    e = out[:, :3] - tn
    loss = 0.5 * np.sum(e * e) / M
    dOut = np.zeros((M, NOUT))
    dOut[:, :3] = e / M
    dOh = r(dOut)
    g = np.zeros(NP)
    g[OW3:OB3] = (dOh.T @ H2).ravel()
    g[OB3:NP] = dOut.sum(axis=0)
    dZ2 = r(np.where(H2 > 0.0, dOh @ W3h, 0.0))
    g[OW2:OB2] = (dZ2.T @ H1).ravel()
    g[OB2:OW3] = dZ2.sum(axis=0)
    dZ1 = r(np.where(H1 > 0.0, dZ2 @ W2h, 0.0))
    g[OW1:OB1] = (dZ1.T @ X).ravel()
    g[OB1:OW2] = dZ1.sum(axis=0)
    return loss, g, out


def random_params(seed: int) -> np.ndarray:
    """He-uniform weights with the padding zero and small random biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NP)
    W1 = rng.uniform(-1, 1, (HID, KIN)) * np.sqrt(6.0 / NF)
    W1[:, NF:] = 0.0
    W3 = rng.uniform(-1, 1, (NOUT, HID)) * np.sqrt(6.0 / HID)
    W3[3:] = 0.0
    p[OW1:OB1] = W1.ravel()
    p[OB1:OW2] = rng.uniform(-0.1, 0.1, HID)
    p[OW2:OB2] = (rng.uniform(-1, 1, (HID, HID)) * np.sqrt(6.0 / HID)).ravel()
    p[OB2:OW3] = rng.uniform(-0.1, 0.1, HID)
    p[OW3:OB3] = W3.ravel()
    p[OB3:OB3 + 3] = rng.uniform(-0.1, 0.1, 3)
    return p.astype(np.float32).astype(np.float64)
