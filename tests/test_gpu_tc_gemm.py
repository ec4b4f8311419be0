"""The network's BF16 GEMM on the 5th-generation tensor cores (tcgen05.mma,
accumulator in tensor memory, operands by TMA) against an exact float64
product of the same bf16 values, and against the mma.sync kernel it replaces.

C = A B^T with FP32 accumulation: each entry differs from the exact sum by at
most about K 2^-24 sum_k |a_ik b_jk| (the bf16 products are exact in FP32);
the bound used is 2^-21 (K + 8) times that sum, room for an accumulation
order or internal rounding of the tensor cores that is not IEEE FP32's.  Shapes: those of the network's training step (batch 4,096: the
forward products, the weight gradients with K = 4,096, the products with K =
16 and 80) and ragged ones (rows, columns and K not multiples of the tile).
"""
import numpy as np
import pytest
import torch

import paper_2102_09964_b300 as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_09964_b300 import build
    build.build()
    P.lib()


SHAPES = [(128, 64, 64), (4096, 256, 80), (4096, 256, 256), (4096, 16, 256), (4096, 256, 16), (16, 256, 4096),
          (256, 256, 4096), (256, 80, 4096), (1000, 200, 72), (136, 72, 8), (5, 3, 24), (300, 64, 136)]


def _case(M, N, K, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Ad, Bd = A.double(), B.double()
    ref = (Ad @ Bd.T).numpy()
    bound = 2.0 ** -21 * (K + 8) * (Ad.abs() @ Bd.abs().T).numpy()
    return A.cuda(), B.cuda(), ref, bound


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_gemm_exact_within_fp32_accumulation(M, N, K, report):
    A, B, ref, bound = _case(M, N, K, M * 7 + N * 3 + K)
    C, err = P.debug_gemm_bf16(A, B, path=0)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    C = C.cpu().numpy().astype(np.float64)
    worst = float(np.max(np.abs(C - ref) / bound))
    report("tcgen05 GEMM |C - exact| / (2^-21 (K + 8) sum|a||b|)", worst, 1.0)
    assert np.all(np.isfinite(C)) and worst <= 1.0, (M, N, K, worst)
    Cm, _ = P.debug_gemm_bf16(A, B, path=1)
    Cm = Cm.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Cm - ref) / bound) <= 1.0
    assert np.max(np.abs(C - Cm) / (2.0 * bound)) <= 1.0


def test_network_gradient_same_on_both_gemm_paths():
    """One training step's loss and gradient through the tcgen05 GEMMs and
    through the mma.sync ones: equal up to FP32 summation order and the BF16
    rounding of activations it can flip (entrywise, with a cap on outliers)."""
    rng = np.random.default_rng(90)
    M = 4096
    feat = torch.as_tensor(rng.normal(size=(M, 65)), dtype=torch.float32, device="cuda")
    theta = torch.as_tensor(rng.normal(size=(M, 3)), dtype=torch.float64, device="cuda")
    net = P.MLP()
    net.init(91, feat, theta)
    out = []
    try:
        for path in (0, 1):
            P.mlp_set_gemm(path)
            g, loss = net.grad(feat, theta)
            out.append((g.cpu().numpy().astype(np.float64), float(loss.item())))
    finally:
        P.mlp_set_gemm(0)
    (g0, l0), (g1, l1) = out
    assert abs(l0 - l1) <= 1e-5 * abs(l1)
    sc = np.abs(g1) + np.sqrt(np.mean(g1 ** 2))
    d = np.abs(g0 - g1) / sc
    assert np.max(d) <= 1e-2 and np.mean(d > 1e-3) <= 1e-2, (np.max(d), np.mean(d > 1e-3))
