"""The allocation-free log-likelihood entry point (pssgp_loglik_noalloc).

Some callers cannot allocate device memory -- a plugin whose host program owns
every device allocation, or a latency-critical loop that must not enter the
driver's allocator -- so they cannot pass a workspace.  For them the library
keeps a fixed scratch array in its own device image.  This file checks,
through the C ABI:
  * two calls in a row on different problems: each equal bit for bit to the
    workspace-based pssgp_loglik on the same inputs (the same kernels run on
    the same scan plan, only the memory differs) and within the
    log-likelihood tolerance of the oracle's sequential filter;
  * a problem exactly at the scratch's size limit is accepted, one step more
    is refused with PSSGP_ESCRATCH before anything is launched;
  * the call is refused while the per-kernel timing diagnostic (which would
    create CUDA events) is on.
It is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2102_09964_b300 as P
import workloads as wl
from oracle import model as om

pytestmark = pytest.mark.gpu

ESCRATCH = -7
EINVAL = -1
SCRATCH_BYTES = 32 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_09964_b300 import build
    build.build()
    oracle.build()
    return P.lib()


def inputs(seed, n_train, n_test):
    s = wl.random_series(seed, n_train, n_test, T=0.01 * (n_train + n_test))
    t = np.concatenate([s.t_train, s.t_test])
    order = np.argsort(t, kind="stable")
    mask = np.concatenate([np.ones(n_train, np.uint8), np.zeros(n_test, np.uint8)])[order]
    y = np.concatenate([s.y_train, np.zeros(n_test)])[order]
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return dev(t[order]), dev(y), dev(mask, torch.uint8)


def noalloc_loglik(lib, m, t, y, mask, R):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    Rd = torch.tensor([R], dtype=torch.float64, device="cuda")
    rc = lib.pssgp_loglik_noalloc(ctypes.byref(m.raw), ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(Rd.data_ptr()), 0, t.numel(),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, float(out.item()), int(st.item())


def largest_n(lib, d):
    """Largest n whose workspace fits the scratch (workspace sizes grow with n)."""
    lo, hi = 1, 1 << 22
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if lib.pssgp_workspace_size(d, mid) <= SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("kind", ["matern32", "rbf"])
def test_noalloc_matches_workspace_entry_point_twice(lib, kind):
    tol = 1e-9 if kind != "rbf" else 1e-6
    m = P.build_model(kind, 0.6, 1.2)
    mo = om.make_model(kind, 0.6, 1.2)
    # two different problems in a row: the second call must not see the first's scratch
    for seed, n_train, n_test in [(11, 9000, 700), (12, 5000, 300)]:
        t, y, mask = inputs(seed, n_train, n_test)
        rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
        assert rc == 0 and st == 0
        ref, ws = P.loglik(m, t, y, mask, 0.02)
        assert P.status(ws) == 0
        assert ll == float(ref.item()), (ll, float(ref.item()))
        tn, yn, mn = t.cpu().numpy(), y.cpu().numpy(), mask.cpu().numpy()
        F, Q = oracle.discretize(mo, tn)
        rll = oracle.kalman_filter(mo, F, Q, yn, mn, 0.02)[4]
        assert abs(ll - rll) <= tol * max(abs(rll), n_train), (ll, rll)


def test_noalloc_at_the_size_limit_and_one_step_over(lib):
    m = P.build_model("rbf", 1.0, 1.0)
    nmax = largest_n(lib, m.d)
    t, y, mask = inputs(14, nmax, 0)
    rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
    assert rc == 0 and st == 0
    ref, ws = P.loglik(m, t, y, mask, 0.02)
    assert ll == float(ref.item())
    t, y, mask = inputs(15, nmax + 1, 0)
    rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
    assert rc == ESCRATCH
    assert np.isnan(ll) and st == -1          # nothing was launched


def test_noalloc_rejects_too_large(lib):
    m = P.build_model("rbf", 1.0, 1.0)
    t, y, mask = inputs(13, 40000, 0)
    rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
    assert rc == ESCRATCH
    assert np.isnan(ll) and st == -1          # nothing was launched


def test_noalloc_refused_while_timing_is_on(lib):
    m = P.build_model("matern32", 1.0, 1.0)
    t, y, mask = inputs(16, 2000, 0)
    P.timing(1)
    try:
        rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
    finally:
        P.timing(0)
    assert rc == EINVAL
    assert np.isnan(ll) and st == -1
    rc, ll, st = noalloc_loglik(lib, m, t, y, mask, 0.02)
    assert rc == 0 and st == 0 and np.isfinite(ll)
