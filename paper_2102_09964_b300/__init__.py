"""pssgp: parallel state-space GP regression on B300 (FP64, sm_103a).

Thin Python binding over the C ABI of ``libpssgp.so`` (declared in
``include/pssgp.h``).  It only marshals arguments: every step of the method
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
current CUDA stream.  There is no CPU fallback: if the shared library is
missing or cannot be loaded, importing the entry points raises.

Method: Corenflos, Zhao, Sarkka, "Temporal Gaussian Process Regression in
Logarithmic Time" -- parallel Kalman filter with missing measurements (Sec. 3),
parallel RTS smoother (supplement, Prop. 2), state-space forms and
discretisation (Sec. 2, 4), merge of prediction times (Sec. 4.3).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpssgp.so")

DMAX = 8
NTAYLOR = 16
MATERN12, MATERN32, MATERN52, RBF = 1, 2, 3, 4
KINDS = {"matern12": MATERN12, "matern32": MATERN32, "matern52": MATERN52, "rbf": RBF}

OK = 0
ERRORS = {-1: "EINVAL", -2: "EDIM", -3: "EKERNEL", -4: "EWORKSPACE", -5: "ECUDA", -6: "EMODEL", -7: "ESCRATCH"}
ENAN, EUNSORTED, ENOTPD, EBATCH = 1, 2, 4, 8


class PssgpKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("order", ctypes.c_int32), ("lengthscale", ctypes.c_double),
                ("variance", ctypes.c_double), ("balance", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PssgpModel(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("G", ctypes.c_double * (DMAX * DMAX)), ("W", ctypes.c_double * (DMAX * DMAX)),
                ("Pinf", ctypes.c_double * (DMAX * DMAX)), ("D", ctypes.c_double * DMAX),
                ("gnorm", ctypes.c_double),
                ("fc", ctypes.c_double * (DMAX * DMAX * NTAYLOR)),
                ("qc", ctypes.c_double * (DMAX * DMAX * NTAYLOR)),
                ("hthr_f", ctypes.c_double * (NTAYLOR + 1)), ("hthr_q", ctypes.c_double * (NTAYLOR + 1)),
                ("hmax", ctypes.c_double), ("companion", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("rsup", ctypes.c_double * (DMAX * DMAX)), ("rlast", ctypes.c_double * (DMAX * DMAX)),
                ("lengthscale", ctypes.c_double), ("variance", ctypes.c_double),
                ("hthr_f32", ctypes.c_double * (NTAYLOR + 1)), ("hthr_q32", ctypes.c_double * (NTAYLOR + 1))]


class PssgpError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libpssgp.so (built by ``paper_2102_09964_b300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PssgpError(f"libpssgp.so not found at {LIB_PATH}; run `python -m paper_2102_09964_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sz = ctypes.c_size_t
        L.pssgp_model_bytes.restype = sz
        L.pssgp_model_build.argtypes = [ctypes.POINTER(PssgpKernel), ctypes.POINTER(PssgpModel)]
        L.pssgp_model_from_sde.argtypes = [i32, vp, vp, dp, vp, i32, ctypes.POINTER(PssgpModel)]
        L.pssgp_workspace_size.argtypes = [i32, i64]
        L.pssgp_workspace_size.restype = sz
        L.pssgp_get_status.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.pssgp_merge.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp, vp, vp, sz, vp]
        L.pssgp_discretize.argtypes = [ctypes.POINTER(PssgpModel), vp, i64, vp, vp, i64, vp, sz, vp]
        L.pssgp_filter.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, vp, vp, i64, vp, vp, sz, vp]
        L.pssgp_smooth.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, i64, i64, vp, vp, vp, vp, vp, sz, vp]
        L.pssgp_loglik.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, vp, vp, sz, vp]
        L.pssgp_loglik_batched.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, vp, vp, vp, vp, i64, vp, vp, sz, vp]
        L.pssgp_fit_workspace_size.restype = sz
        L.pssgp_fit_workspace_size.argtypes = [i32, i64, i32]
        L.pssgp_fit_batched.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, vp, vp, vp, i64, vp, vp, vp,
                                        ctypes.POINTER(FitOptions), vp, sz, vp, ctypes.POINTER(i32)]
        L.pssgp_simulate_prior.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, vp, ctypes.c_uint64, dp, vp, vp,
                                           vp, vp]
        L.pssgp_features.argtypes = [vp, i32, vp, vp, vp, vp]
        L.pssgp_mlp_state_bytes.restype = sz
        L.pssgp_mlp_workspace_size.restype = sz
        L.pssgp_mlp_workspace_size.argtypes = [i32]
        L.pssgp_mlp_init.argtypes = [vp, ctypes.c_uint64, vp, i64, vp, vp]
        L.pssgp_mlp_set_params.argtypes = [vp, vp, vp, vp]
        L.pssgp_mlp_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, sz, vp]
        L.pssgp_mlp_adam.argtypes = [vp, vp, ctypes.c_float, i32, vp]
        L.pssgp_mlp_predict.argtypes = [vp, vp, i32, vp, vp, sz, vp]
        L.pssgp_workspace_size_grad.restype = sz
        L.pssgp_workspace_size_grad.argtypes = [i32, i64]
        L.pssgp_loglik_grad.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, vp, vp, vp, sz, vp]
        L.pssgp_loglik_grad_batched.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, vp, vp, vp, vp, i64, vp, vp,
                                                vp, sz, vp]
        L.pssgp_predict.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, i64, vp, i64, dp, vp, vp, vp, vp, sz, vp]
        L.pssgp_predict_host.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, i64, vp, i64, dp, vp, vp, vp, vp, sz,
                                         vp]
        L.pssgp_predict_host_workspace_size.restype = sz
        L.pssgp_predict_host_workspace_size.argtypes = [i32, i64, i64]
        L.pssgp_debug_filter_aggregates.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i64, i32,
                                                    vp, vp, ctypes.POINTER(i32), vp, sz, vp]
        L.pssgp_fp64_fma_rate.argtypes = [ctypes.POINTER(dp)]
        L.pssgp_timing.argtypes = [i32, vp, vp, i32]
        L.pssgp_set_warps_per_sm.argtypes = [i32]
        L.pssgp_tune_set.argtypes = [i32, i32]
        L.pssgp_tune_get.argtypes = [i32]
        L.pssgp_autotune_loglik_batched.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, vp, vp, vp, vp, i64, vp,
                                                    vp, sz, vp, i32, ctypes.POINTER(i32),
                                                    ctypes.POINTER(ctypes.c_float)]
        L.pssgp_graph_begin.argtypes = [vp]
        L.pssgp_graph_end.argtypes = [vp, ctypes.POINTER(vp)]
        L.pssgp_graph_launch.argtypes = [vp, vp]
        L.pssgp_graph_destroy.argtypes = [vp]
        L.pssgp_loglik_noalloc.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, vp, vp, vp]
        L.pssgp_split_agg_doubles.argtypes = [i32, i32]
        L.pssgp_split_agg_doubles.restype = i32
        L.pssgp_split_filter_reduce.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, dp, dp, i32,
                                                vp, vp, sz, vp]
        L.pssgp_split_filter_finish.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, vp, vp, i32, i64, dp, i32, vp,
                                                i32, i32, vp, vp, i64, vp, vp, sz, vp]
        L.pssgp_split_smooth_reduce.argtypes = [ctypes.POINTER(PssgpModel), i64, vp, vp, sz, vp]
        L.pssgp_split_smooth_finish.argtypes = [ctypes.POINTER(PssgpModel), i64, i64, vp, i32, i32, vp, vp, vp, vp,
                                                vp, sz, vp]
        L.pssgp_split_grad_mean_reduce.argtypes = [ctypes.POINTER(PssgpModel), i64, vp, vp, sz, vp]
        L.pssgp_split_grad_mean_finish.argtypes = [ctypes.POINTER(PssgpModel), i64, vp, i32, i32, vp, vp, sz, vp]
        L.pssgp_split_grad_finish.argtypes = [ctypes.POINTER(PssgpModel), vp, i32, i64, vp, i32, i32, vp, vp, sz,
                                              vp]
        L.pssgp_predict_batched_workspace_size.restype = sz
        L.pssgp_predict_batched_workspace_size.argtypes = [i32, i64, i64, i32]
        L.pssgp_predict_batched.argtypes = [ctypes.POINTER(PssgpModel), vp, vp, i32, vp, vp, vp, i64, vp, i64, vp, vp,
                                            vp, vp, sz, vp]
        L.pssgp_mlp_set_gemm.argtypes = [i32]
        L.pssgp_debug_gemm_bf16.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp]
        L.pssgp_timing_name.argtypes = [i32]
        L.pssgp_timing_name.restype = ctypes.c_char_p
        if L.pssgp_model_bytes() != ctypes.sizeof(PssgpModel):
            raise PssgpError("pssgp_model layout mismatch between libpssgp.so and the binding")
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise PssgpError(f"{what} failed: {ERRORS.get(rc, rc)}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# PSSGP_NAN_FILL=1: every output and workspace the binding allocates is filled
# with 0xFF bytes (NaN for floating point, -1 for integers) before the call,
# so that an entry the library should write but does not is visible.
_NAN_FILL = os.environ.get("PSSGP_NAN_FILL", "0") not in ("", "0")


def _empty(*size, dtype, device):
    t = torch.empty(*size, dtype=dtype, device=device)
    if _NAN_FILL and t.numel() > 0:
        t.view(torch.uint8).fill_(0xFF)
    return t


@dataclass
class Model:
    """A built state-space model (host struct handed to every call)."""
    raw: PssgpModel

    @property
    def d(self) -> int:
        return int(self.raw.d)

    @property
    def D(self):
        return [self.raw.D[i] for i in range(self.d)]

    def matrix(self, name: str):
        import numpy as np
        a = getattr(self.raw, name)
        d = self.d
        return np.array([a[i] for i in range(d * d)]).reshape(d, d)


def build_model(kind: str, lengthscale: float, variance: float, order: int = 6, balance: bool = True) -> Model:
    """Kernel -> SDE -> P_inf -> balancing -> discretisation tables (host, O(1))."""
    k = PssgpKernel(KINDS[kind], int(order), float(lengthscale), float(variance), int(bool(balance)), 0)
    m = PssgpModel()
    _check(lib().pssgp_model_build(ctypes.byref(k), ctypes.byref(m)), "pssgp_model_build")
    return Model(m)


def model_from_sde(G, L, q: float, H, balance: bool = True) -> Model:
    import numpy as np
    G = np.ascontiguousarray(G, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64).ravel()
    H = np.ascontiguousarray(H, dtype=np.float64).ravel()
    m = PssgpModel()
    rc = lib().pssgp_model_from_sde(G.shape[0], G.ctypes.data, L.ctypes.data, float(q), H.ctypes.data,
                                    int(bool(balance)), ctypes.byref(m))
    _check(rc, "pssgp_model_from_sde")
    return Model(m)


def workspace_size(d: int, n: int) -> int:
    return int(lib().pssgp_workspace_size(int(d), int(n)))


def workspace(d: int, n: int, device="cuda", extra: int = 0) -> torch.Tensor:
    """A device workspace of the size the library asks for (torch allocations
    are 256-byte aligned)."""
    return _empty(workspace_size(d, n) + int(extra), dtype=torch.uint8, device=device)


def workspace_grad(d: int, n: int, device="cuda") -> torch.Tensor:
    """A device workspace for the gradient entry points."""
    return _empty(int(lib().pssgp_workspace_size_grad(int(d), int(n))), dtype=torch.uint8, device=device)


def status(ws: torch.Tensor) -> int:
    """Device status word of the last call on `ws` (synchronises the stream)."""
    v = ctypes.c_int32(0)
    _check(lib().pssgp_get_status(_ptr(ws), _stream(), ctypes.byref(v)), "pssgp_get_status")
    return int(v.value)


def _f64(x, dev):
    return torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous()


def merge(t_train, y_train, t_test, ws=None):
    dev = t_train.device
    N, M = t_train.numel(), t_test.numel()
    n = N + M
    t = _empty(n, dtype=torch.float64, device=dev)
    y = _empty(n, dtype=torch.float64, device=dev)
    mask = _empty(n, dtype=torch.uint8, device=dev)
    tpos = _empty(max(M, 1), dtype=torch.int64, device=dev)
    ws = ws if ws is not None else _empty(256, dtype=torch.uint8, device=dev)
    rc = lib().pssgp_merge(_ptr(t_train), _ptr(y_train), N, _ptr(t_test), M, _ptr(t), _ptr(y), _ptr(mask),
                           _ptr(tpos), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_merge")
    return t, y, mask, tpos[:M], ws


def discretize(model: Model, t, ws=None):
    """F (d*d x n, entry-major) and Q (packed x n)."""
    d, n = model.d, t.numel()
    F = _empty(d * d, n, dtype=torch.float64, device=t.device)
    Q = _empty(d * (d + 1) // 2, n, dtype=torch.float64, device=t.device)
    ws = ws if ws is not None else _empty(256, dtype=torch.uint8, device=t.device)
    rc = lib().pssgp_discretize(ctypes.byref(model.raw), _ptr(t), n, _ptr(F), _ptr(Q), n, _ptr(ws), ws.numel(),
                                _stream())
    _check(rc, "pssgp_discretize")
    return F, Q, ws


def filter(model: Model, t, y, mask, R, ws=None, outputs=True, loglik=True):
    """Parallel Kalman filter; returns (xf, Pf, loglik tensor, ws)."""
    d, n = model.d, t.numel()
    dev = t.device
    R = _f64(R, dev).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    ws = ws if ws is not None else workspace(d, n, dev)
    xf = _empty(d, n, dtype=torch.float64, device=dev) if outputs else None
    Pf = _empty(d * (d + 1) // 2, n, dtype=torch.float64, device=dev) if outputs else None
    ll = _empty(1, dtype=torch.float64, device=dev) if loglik else None
    rc = lib().pssgp_filter(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), per, n, _ptr(xf),
                            _ptr(Pf), n, _ptr(ll), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_filter")
    return xf, Pf, ll, ws


def smooth(model: Model, t, xf, Pf, ws=None, states=False):
    """Parallel RTS smoother from filter outputs; returns (f_mean, f_var, xs, Ps, ws)."""
    d, n = model.d, t.numel()
    dev = t.device
    ws = ws if ws is not None else workspace(d, n, dev)
    fm = _empty(n, dtype=torch.float64, device=dev)
    fv = _empty(n, dtype=torch.float64, device=dev)
    xs = _empty(d, n, dtype=torch.float64, device=dev) if states else None
    Ps = _empty(d * (d + 1) // 2, n, dtype=torch.float64, device=dev) if states else None
    rc = lib().pssgp_smooth(ctypes.byref(model.raw), _ptr(t), _ptr(xf), _ptr(Pf), n, n, _ptr(fm), _ptr(fv),
                            _ptr(xs), _ptr(Ps), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_smooth")
    return fm, fv, xs, Ps, ws


def loglik(model: Model, t, y, mask, R, ws=None):
    d, n = model.d, t.numel()
    dev = t.device
    R = _f64(R, dev).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    ws = ws if ws is not None else workspace(d, n, dev)
    ll = _empty(1, dtype=torch.float64, device=dev)
    rc = lib().pssgp_loglik(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), per, n, _ptr(ll),
                            _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_loglik")
    return ll, ws


def loglik_batched(model: Model, offsets, params, t, y, mask, ws=None, out=None):
    """Log marginal likelihoods of B series in one pass.  offsets: int64[B+1]
    (series s = steps offsets[s]..offsets[s+1]-1 of t, y, mask); params:
    float64[B, 3] = (lengthscale, variance, noise variance) per series; model:
    the kernel family, built at any hyperparameters.  Returns (loglik[B], ws)."""
    d, n = model.d, t.numel()
    dev = t.device
    B = offsets.numel() - 1
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise TypeError("offsets must be a contiguous int64 tensor")
    params = _f64(params, dev).reshape(-1)
    if params.numel() != 3 * B:
        raise ValueError("params must hold 3 values per series")
    ws = ws if ws is not None else workspace(d, n, dev)
    ll = out if out is not None else _empty(B, dtype=torch.float64, device=dev)
    rc = lib().pssgp_loglik_batched(ctypes.byref(model.raw), _ptr(offsets), B, _ptr(params), _ptr(t), _ptr(y),
                                    _ptr(mask), n, _ptr(ll), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_loglik_batched")
    return ll, ws


def loglik_grad(model: Model, t, y, mask, R, ws=None):
    """Log-likelihood of one series and its gradient with respect to
    (log lengthscale, log variance, log noise variance) by the adjoint scans.
    R: scalar or per step (the noise derivative scales every R_k).
    Returns (loglik[1], grad[3], ws)."""
    d, n = model.d, t.numel()
    dev = t.device
    R = _f64(R, dev).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    ws = ws if ws is not None else workspace_grad(d, n, dev)
    ll = _empty(1, dtype=torch.float64, device=dev)
    g = _empty(3, dtype=torch.float64, device=dev)
    rc = lib().pssgp_loglik_grad(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), per, n, _ptr(ll),
                                 _ptr(g), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_loglik_grad")
    return ll, g, ws


def loglik_grad_batched(model: Model, offsets, params, t, y, mask, ws=None, out=None):
    """Log-likelihoods of B series and their gradients with respect to each
    series' (log lengthscale, log variance, log noise variance).  Arguments
    as loglik_batched.  Returns (loglik[B], grad[B, 3], ws)."""
    d, n = model.d, t.numel()
    dev = t.device
    B = offsets.numel() - 1
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise TypeError("offsets must be a contiguous int64 tensor")
    params = _f64(params, dev).reshape(-1)
    if params.numel() != 3 * B:
        raise ValueError("params must hold 3 values per series")
    ws = ws if ws is not None else workspace_grad(d, n, dev)
    if out is None:
        out = (_empty(B, dtype=torch.float64, device=dev), _empty(B, 3, dtype=torch.float64, device=dev))
    ll, g = out
    rc = lib().pssgp_loglik_grad_batched(ctypes.byref(model.raw), _ptr(offsets), B, _ptr(params), _ptr(t), _ptr(y),
                                         _ptr(mask), n, _ptr(ll), _ptr(g), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_loglik_grad_batched")
    return ll, g, ws


class FitOptions(ctypes.Structure):
    """pssgp_fit_options."""
    _fields_ = [("max_iter", ctypes.c_int32), ("patience", ctypes.c_int32), ("tol", ctypes.c_double),
                ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("check_every", ctypes.c_int32), ("method", ctypes.c_int32)]


FIT_ADAM, FIT_LBFGS = 0, 1


def fit_batched(model: Model, offsets, t, y, mask, theta0, max_iter=2000, patience=10, tol=1e-7, lr=0.05,
                beta1=0.9, beta2=0.999, eps=1e-8, check_every=1, ws=None, method="adam"):
    """Adam (method="adam") or L-BFGS (method="lbfgs") fit of every series'
    (log l, log s2, log R) on its exact log marginal likelihood (native driver).  offsets: host int64 array [B+1];
    t, y, mask: device arrays; theta0: [B, 3] start (log values).
    Returns (theta[B, 3], loglik[B], iters[B], iterations_run)."""
    import numpy as np
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    B = offs.size - 1
    n = t.numel()
    dev = t.device
    theta = _f64(theta0, dev).reshape(B, 3).clone()
    ll = _empty(B, dtype=torch.float64, device=dev)
    it = _empty(B, dtype=torch.int32, device=dev)
    if ws is None:
        ws = _empty(int(lib().pssgp_fit_workspace_size(model.d, n, B)), dtype=torch.uint8, device=dev)
    o = FitOptions(int(max_iter), int(patience), float(tol), float(lr), float(beta1), float(beta2), float(eps),
                   int(check_every), {"adam": FIT_ADAM, "lbfgs": FIT_LBFGS}[method])
    nrun = ctypes.c_int32(0)
    rc = lib().pssgp_fit_batched(ctypes.byref(model.raw), offs.ctypes.data_as(ctypes.c_void_p), B, _ptr(t), _ptr(y),
                                 _ptr(mask), n, _ptr(theta), _ptr(ll), _ptr(it), ctypes.byref(o), _ptr(ws),
                                 ws.numel(), _stream(), ctypes.byref(nrun))
    _check(rc, "pssgp_fit_batched")
    return theta, ll, it, int(nrun.value)


class BatchedLogLik(torch.autograd.Function):
    """ll[B] = log marginal likelihoods of B series as a function of their
    log hyperparameters theta[B, 3] = (log lengthscale, log variance,
    log noise variance); the backward pass is the adjoint scans' gradient
    (computed together with the forward values in one library call)."""

    @staticmethod
    def forward(ctx, theta, model, offsets, t, y, mask, ws):
        params = torch.exp(theta.detach()).contiguous()
        ll, g, _ = loglik_grad_batched(model, offsets, params, t, y, mask, ws=ws)
        ctx.save_for_backward(g)
        return ll

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout[:, None] * g, None, None, None, None, None, None


def batched_loglik(theta, model: Model, offsets, t, y, mask, ws=None):
    """Differentiable batched log-likelihood (see BatchedLogLik)."""
    if ws is None:
        ws = workspace_grad(model.d, t.numel(), t.device)
    return BatchedLogLik.apply(theta, model, offsets, t, y, mask, ws)


def predict(model: Model, t_train, y_train, t_test, R: float, ws=None, out=None, with_loglik=True):
    """Fused merge + filter + smoother + gather.  Returns (mean, var, loglik, ws)."""
    N, M = t_train.numel(), t_test.numel()
    dev = t_train.device
    ws = ws if ws is not None else workspace(model.d, N + M, dev)
    if out is None:
        out = (_empty(M, dtype=torch.float64, device=dev), _empty(M, dtype=torch.float64, device=dev),
               _empty(1, dtype=torch.float64, device=dev))
    mean, var, ll = out
    rc = lib().pssgp_predict(ctypes.byref(model.raw), _ptr(t_train), _ptr(y_train), N, _ptr(t_test), M, float(R),
                             _ptr(mean), _ptr(var), _ptr(ll) if with_loglik else None, _ptr(ws), ws.numel(),
                             _stream())
    _check(rc, "pssgp_predict")
    return mean, var, ll, ws


def predict_batched(model: Model, train_offsets, test_offsets, params, t_train, y_train, t_test, ws=None,
                    with_loglik=True, out=None):
    """Posterior mean and variance at the prediction times of B series, and
    each series' log-likelihood, in one pass (pssgp_predict_batched).  Offsets:
    device int64[B + 1] into the training (t_train, y_train) and prediction
    (t_test) arrays; params: device float64[B, 3] (lengthscale, variance,
    noise variance); out: optional (mean[M], var[M], loglik[B]) buffers
    (needed inside a Graph capture).  Returns (mean, var, loglik or None, ws)."""
    dev = t_train.device if t_train.numel() else t_test.device
    B = train_offsets.numel() - 1
    N, M = t_train.numel(), t_test.numel()
    for o in (train_offsets, test_offsets):
        if o.dtype != torch.int64 or not o.is_contiguous():
            raise PssgpError("offsets must be contiguous int64")
    params = params.contiguous()
    if ws is None:
        ws = _empty(int(lib().pssgp_predict_batched_workspace_size(model.d, N, M, B)), dtype=torch.uint8,
                    device=dev)
    if out is not None:
        mean, var, ll = out
    else:
        mean = _empty(M, dtype=torch.float64, device=dev)
        var = _empty(M, dtype=torch.float64, device=dev)
        ll = _empty(B, dtype=torch.float64, device=dev) if with_loglik else None
    rc = lib().pssgp_predict_batched(ctypes.byref(model.raw), _ptr(train_offsets), _ptr(test_offsets), B,
                                     _ptr(params), _ptr(t_train), _ptr(y_train), N, _ptr(t_test), M, _ptr(mean),
                                     _ptr(var), _ptr(ll), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_predict_batched")
    return mean, var, ll, ws


def predict_host(model: Model, t_train, y_train, t_test, R: float, out, ws=None, stream=None):
    """pssgp_predict from and to host tensors (page-locked for overlap):
    out = (mean[M], var[M], loglik[1]) host float64 tensors.  Asynchronous on
    `stream` (default: the current stream); returns the workspace."""
    N, M = t_train.numel(), t_test.numel()
    if ws is None:
        ws = _empty(int(lib().pssgp_predict_host_workspace_size(model.d, N, M)), dtype=torch.uint8,
                         device="cuda")
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    mean, var, ll = out
    rc = lib().pssgp_predict_host(ctypes.byref(model.raw), _ptr(t_train), _ptr(y_train), N, _ptr(t_test), M,
                                  float(R), _ptr(mean), _ptr(var), _ptr(ll), _ptr(ws), ws.numel(), st)
    _check(rc, "pssgp_predict_host")
    return ws


# ---------------------------------------------------------------------------
# one long series split in time chunks over several GPUs (calls of one rank;
# the exchange between them is in paper_2102_09964_b300.split)
# ---------------------------------------------------------------------------
def split_agg_doubles(d: int, smoother: bool) -> int:
    return int(lib().pssgp_split_agg_doubles(int(d), int(bool(smoother))))


def _split_mode(smoother, grad):
    return 2 if grad else int(bool(smoother))


def split_filter_reduce(model: Model, t, y, mask, R, t_prev: float, t_next: float, ws, smoother=True, agg=None,
                        grad=False):
    """This chunk's filter aggregate (device float64[nf]); ws carries state to
    split_filter_finish (which must get the same t_next, smoother and grad).
    grad: the adjoint pass of the gradient follows (ws from workspace_grad)."""
    d, n = model.d, t.numel()
    R = _f64(R, t.device).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    agg = agg if agg is not None else _empty(split_agg_doubles(d, False), dtype=torch.float64, device=t.device)
    rc = lib().pssgp_split_filter_reduce(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), per, n,
                                         float(t_prev), float(t_next), _split_mode(smoother, grad), _ptr(agg), _ptr(ws),
                                         ws.numel(), _stream())
    _check(rc, "pssgp_split_filter_reduce")
    return agg


def split_filter_finish(model: Model, t, y, mask, R, t_next: float, aggs, rank: int, ws, smoother=True,
                        outputs=True, grad=False):
    """Filter outputs of this chunk given every chunk's aggregate (aggs: device
    float64[G, nf] in rank order), and with smoother its smoother elements;
    returns (xf, Pf, loglik[1]) with xf, Pf None unless outputs."""
    d, n = model.d, t.numel()
    dev = t.device
    R = _f64(R, dev).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    aggs = aggs.contiguous()
    xf = _empty(d, n, dtype=torch.float64, device=dev) if outputs else None
    Pf = _empty(d * (d + 1) // 2, n, dtype=torch.float64, device=dev) if outputs else None
    ll = _empty(1, dtype=torch.float64, device=dev)
    rc = lib().pssgp_split_filter_finish(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), per, n,
                                         float(t_next), _split_mode(smoother, grad), _ptr(aggs), aggs.shape[0],
                                         int(rank),
                                         _ptr(xf), _ptr(Pf), n, _ptr(ll), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_split_filter_finish")
    return xf, Pf, ll


def split_smooth_reduce(model: Model, n: int, ws, agg=None, device="cuda"):
    """This chunk's smoother aggregate (device float64[ns]), after
    split_filter_finish with the smoother."""
    agg = agg if agg is not None else _empty(split_agg_doubles(model.d, True), dtype=torch.float64, device=device)
    rc = lib().pssgp_split_smooth_reduce(ctypes.byref(model.raw), int(n), _ptr(agg), _ptr(ws), ws.numel(),
                                         _stream())
    _check(rc, "pssgp_split_smooth_reduce")
    return agg


def split_smooth_finish(model: Model, n: int, aggs, rank: int, ws, device="cuda", states=False):
    """Smoother outputs of this chunk given every chunk's smoother aggregate;
    returns (f_mean, f_var, xs, Ps) with xs, Ps None unless states."""
    d = model.d
    aggs = aggs.contiguous()
    fm = _empty(n, dtype=torch.float64, device=device)
    fv = _empty(n, dtype=torch.float64, device=device)
    xs = _empty(d, n, dtype=torch.float64, device=device) if states else None
    Ps = _empty(d * (d + 1) // 2, n, dtype=torch.float64, device=device) if states else None
    rc = lib().pssgp_split_smooth_finish(ctypes.byref(model.raw), n, n, _ptr(aggs), aggs.shape[0], int(rank),
                                         _ptr(fm), _ptr(fv), _ptr(xs), _ptr(Ps), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_split_smooth_finish")
    return fm, fv, xs, Ps


def split_grad_mean_reduce(model: Model, n: int, ws, device="cuda"):
    """This chunk's mean-adjoint aggregate (device float64[ns]), after
    split_filter_finish with grad."""
    agg = _empty(split_agg_doubles(model.d, True), dtype=torch.float64, device=device)
    _check(lib().pssgp_split_grad_mean_reduce(ctypes.byref(model.raw), int(n), _ptr(agg), _ptr(ws), ws.numel(),
                                              _stream()), "pssgp_split_grad_mean_reduce")
    return agg


def split_grad_mean_finish(model: Model, n: int, aggs, rank: int, ws, device="cuda"):
    """Given every chunk's mean-adjoint aggregate (device float64[G, ns]):
    this chunk's covariance-adjoint aggregate (device float64[ns])."""
    aggs = aggs.contiguous()
    agg = _empty(split_agg_doubles(model.d, True), dtype=torch.float64, device=device)
    _check(lib().pssgp_split_grad_mean_finish(ctypes.byref(model.raw), int(n), _ptr(aggs), aggs.shape[0],
                                              int(rank), _ptr(agg), _ptr(ws), ws.numel(), _stream()),
           "pssgp_split_grad_mean_finish")
    return agg


def split_grad_finish(model: Model, n: int, R, aggs, rank: int, ws, device="cuda"):
    """Given every chunk's covariance-adjoint aggregate: this chunk's terms of
    the gradient (device float64[3]); R as in split_filter_reduce."""
    R = _f64(R, device).reshape(-1)
    per = 1 if R.numel() == n and n > 1 else 0
    aggs = aggs.contiguous()
    g = _empty(3, dtype=torch.float64, device=device)
    _check(lib().pssgp_split_grad_finish(ctypes.byref(model.raw), _ptr(R), per, int(n), _ptr(aggs), aggs.shape[0],
                                         int(rank), _ptr(g), _ptr(ws), ws.numel(), _stream()),
           "pssgp_split_grad_finish")
    return g


def debug_filter_aggregates(model: Model, t, y, mask, R, lanes: int = 0):
    """Level-0 chunk aggregates (A, b, C, eta, J) per lane, in SDE coordinates,
    and each chunk's first step (host numpy arrays)."""
    import numpy as np
    d, n = model.d, t.numel()
    dev = t.device
    R = _f64(R, dev).reshape(-1)[:1]
    lanes_req = lanes
    # room for the per-lane debug copy after the regular workspace
    lanes_max = max(lanes_req, 148 * 4 * 32, 128)
    ws = workspace(d, n, dev, extra=lanes_max * (2 * d * d + 3 * d) * 8 + 4096)
    nf = 3 * d * d + 2 * d
    agg = np.zeros((lanes_max + 128, nf))
    first = np.zeros(lanes_max + 128, dtype=np.int64)
    used = ctypes.c_int32(0)
    rc = lib().pssgp_debug_filter_aggregates(ctypes.byref(model.raw), _ptr(t), _ptr(y), _ptr(mask), _ptr(R), n,
                                             int(lanes_req), agg.ctypes.data, first.ctypes.data,
                                             ctypes.byref(used), _ptr(ws), ws.numel(), _stream())
    _check(rc, "pssgp_debug_filter_aggregates")
    P0 = used.value
    out = []
    for c in range(P0):
        a = agg[c]
        out.append((a[:d * d].reshape(d, d), a[d * d:d * d + d], a[d * d + d:2 * d * d + d].reshape(d, d),
                    a[2 * d * d + d:2 * d * d + 2 * d], a[2 * d * d + 2 * d:].reshape(d, d)))
    return out, first[:P0], status(ws)


def mlp_set_gemm(path: int):
    """0: the network's GEMMs on tcgen05 (default); 1: the mma.sync baseline."""
    _check(lib().pssgp_mlp_set_gemm(int(path)), "pssgp_mlp_set_gemm")


def debug_gemm_bf16(A, B, path: int = 0):
    """C = A B^T (A: bf16 [M, K], B: bf16 [N, K], device) in float32 with the
    chosen GEMM; returns (C, err) with err the kernel's timeout flag."""
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = _empty(M, N, dtype=torch.float32, device=A.device)
    err = torch.full((1,), -1, dtype=torch.int32, device=A.device)
    _check(lib().pssgp_debug_gemm_bf16(_ptr(A), _ptr(B), M, N, K, _ptr(C), int(path), _ptr(err), _stream()),
           "pssgp_debug_gemm_bf16")
    return C, err


def fp64_fma_rate() -> float:
    v = ctypes.c_double(0.0)
    _check(lib().pssgp_fp64_fma_rate(ctypes.byref(v)), "pssgp_fp64_fma_rate")
    return float(v.value)


def timing(mode: int):
    """Per-kernel event timing: timing(1) enable+reset, timing(0) disable,
    timing(2) -> {kernel name: (total ms, launches)}."""
    import numpy as np
    ms = np.zeros(16)
    cnt = np.zeros(16, dtype=np.int64)
    _check(lib().pssgp_timing(int(mode), ms.ctypes.data if mode == 2 else None,
                              cnt.ctypes.data if mode == 2 else None, 16), "pssgp_timing")
    if mode != 2:
        return None
    out = {}
    for i in range(16):
        name = lib().pssgp_timing_name(i).decode()
        if name and cnt[i] > 0:
            out[name] = (float(ms[i]), int(cnt[i]))
    return out


def set_warps_per_sm(w: int):
    """Scan tuning knob for every state dimension (4, 8, 12 or 16 warps per SM)."""
    _check(lib().pssgp_set_warps_per_sm(int(w)), "pssgp_set_warps_per_sm")


def tune_set(d: int, w: int):
    """Scan tuning knob for state dimension d (4, 8, 12 or 16 warps per SM)."""
    _check(lib().pssgp_tune_set(int(d), int(w)), "pssgp_tune_set")


def tune_get(d: int) -> int:
    w = lib().pssgp_tune_get(int(d))
    _check(min(w, 0), "pssgp_tune_get")
    return w


def _tune_key(d: int, n: int, B: int) -> str:
    import math
    name = torch.cuda.get_device_name()
    return f"{name}|loglik_batched|d={d}|n=2^{round(math.log2(max(n, 1)))}|B=2^{round(math.log2(max(B, 1)))}"


def autotune_loglik_batched(model: Model, offsets, params, t, y, mask, ws=None, out=None, reps: int = 3,
                            cache: str | None = None):
    """Pick the scan lane count for this batch shape by timing every candidate
    (native autotuner), and apply it for model.d.  With `cache` (a JSON file),
    a stored choice for the same device, d and size class is applied without
    timing, and new choices are stored.  Returns (warps_per_sm, ms or None)."""
    import json
    import os
    d, n = model.d, t.numel()
    B = offsets.numel() - 1
    key = _tune_key(d, n, B)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            tune_set(d, int(table[key]["warps_per_sm"]))
            return int(table[key]["warps_per_sm"]), None
    ws = ws if ws is not None else workspace(d, n, t.device)
    ll = out if out is not None else _empty(B, dtype=torch.float64, device=t.device)
    params = _f64(params, t.device).reshape(-1)
    w = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    rc = lib().pssgp_autotune_loglik_batched(ctypes.byref(model.raw), _ptr(offsets), B, _ptr(params), _ptr(t),
                                             _ptr(y), _ptr(mask), n, _ptr(ll), _ptr(ws), ws.numel(), _stream(),
                                             int(reps), ctypes.byref(w), ctypes.byref(ms))
    _check(rc, "pssgp_autotune_loglik_batched")
    if cache:
        table[key] = {"warps_per_sm": int(w.value), "ms": float(ms.value)}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return int(w.value), float(ms.value)


class Graph:
    """A sequence of library calls recorded once into a CUDA graph and replayed
    with one launch (native stream capture).  Use on a non-default stream:

        g = Graph(stream)
        with g:
            loglik_batched(..., ws=ws, out=ll)     # buffers allocated beforehand
        g.launch()                                  # replays all recorded launches
    """

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._h = ctypes.c_void_p(None)
        self._ctx = None

    def __enter__(self):
        self._ctx = torch.cuda.stream(self.stream)
        self._ctx.__enter__()
        _check(lib().pssgp_graph_begin(ctypes.c_void_p(self.stream.cuda_stream)), "pssgp_graph_begin")
        return self

    def __exit__(self, exc_type, exc, tb):
        h = ctypes.c_void_p(None)
        rc = lib().pssgp_graph_end(ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self._ctx.__exit__(exc_type, exc, tb)
        if exc_type is None:
            _check(rc, "pssgp_graph_end")
            self._h = h
        return False

    def launch(self):
        """Enqueue the recorded work on the graph's stream and make the current
        stream wait for it."""
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        _check(lib().pssgp_graph_launch(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "pssgp_graph_launch")
        cur.wait_stream(self.stream)

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            try:
                lib().pssgp_graph_destroy(self._h)
            except Exception:
                pass
            self._h = ctypes.c_void_p(None)


# ---------------------------------------------------------------------------
# learned initialisation: prior simulation, features, the network
# ---------------------------------------------------------------------------
NFEAT = 65


def simulate_prior(model: Model, offsets, params, seed: int, spacing: float = 0.01):
    """Series drawn from the prior of the model's family at per-series
    (lengthscale, variance, noise) params[B, 3]; offsets: device int64[B+1].
    Returns (t, y) device float64 arrays of length offsets[-1]."""
    dev = offsets.device
    B = offsets.numel() - 1
    n = int(offsets[-1].item())
    params = _f64(params, dev).reshape(-1)
    t = _empty(max(n, 1), dtype=torch.float64, device=dev)
    y = _empty(max(n, 1), dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = lib().pssgp_simulate_prior(ctypes.byref(model.raw), _ptr(offsets), B, _ptr(params), int(seed),
                                    float(spacing), _ptr(t), _ptr(y), _ptr(st), _stream())
    _check(rc, "pssgp_simulate_prior")
    return t[:n], y[:n], st


def features(offsets, t, y, out=None):
    """The 65 log-periodogram features of every series (device float32[B, 65])."""
    B = offsets.numel() - 1
    f = out if out is not None else _empty(B, NFEAT, dtype=torch.float32, device=t.device)
    _check(lib().pssgp_features(_ptr(offsets), B, _ptr(t), _ptr(y), _ptr(f), _stream()), "pssgp_features")
    return f


class MLP:
    """The initialisation network (state in one device buffer, see pssgp.h)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.state = torch.zeros(int(lib().pssgp_mlp_state_bytes()), dtype=torch.uint8, device=self.device)
        self.nparam = int(lib().pssgp_mlp_param_count())
        self.step = 0
        self._ws = {}

    def ws(self, rows: int):
        if rows not in self._ws:
            self._ws[rows] = _empty(int(lib().pssgp_mlp_workspace_size(int(rows))), dtype=torch.uint8,
                                         device=self.device)
        return self._ws[rows]

    def init(self, seed: int, feat, theta):
        _check(lib().pssgp_mlp_init(_ptr(self.state), int(seed), _ptr(feat), feat.shape[0], _ptr(theta),
                                    _stream()), "pssgp_mlp_init")
        self.step = 0

    def set_params(self, params, norm):
        params = torch.as_tensor(params, dtype=torch.float32, device=self.device).contiguous()
        norm = torch.as_tensor(norm, dtype=torch.float32, device=self.device).contiguous()
        _check(lib().pssgp_mlp_set_params(_ptr(self.state), _ptr(params), _ptr(norm), _stream()),
               "pssgp_mlp_set_params")
        self.step = 0

    def grad(self, feat, theta, grad=None, loss=None, out=None):
        rows = feat.shape[0]
        g = grad if grad is not None else _empty(self.nparam, dtype=torch.float32, device=self.device)
        ls = loss if loss is not None else _empty(1, dtype=torch.float32, device=self.device)
        ws = self.ws(rows)
        _check(lib().pssgp_mlp_grad(_ptr(self.state), _ptr(feat), _ptr(theta), rows, _ptr(g), _ptr(ls), _ptr(out),
                                    _ptr(ws), ws.numel(), _stream()), "pssgp_mlp_grad")
        return g, ls

    def adam(self, grad, lr: float):
        self.step += 1
        _check(lib().pssgp_mlp_adam(_ptr(self.state), _ptr(grad), float(lr), self.step, _stream()), "pssgp_mlp_adam")

    def train(self, feat, theta, epochs: int, batch: int = 4096, lr: float = 1e-3, lr_final: float = 1e-4):
        """Adam on consecutive minibatches (the rows are i.i.d. draws, so a
        fixed order is a random one); cosine-free geometric decay of the step
        from lr to lr_final.  Returns the loss of every step (device)."""
        rows = feat.shape[0]
        nb = rows // batch
        g = _empty(self.nparam, dtype=torch.float32, device=self.device)
        losses = _empty(max(epochs * nb, 1), dtype=torch.float32, device=self.device)
        total = epochs * nb
        for e in range(epochs):
            for b in range(nb):
                i = e * nb + b
                a = b * batch
                self.grad(feat[a:a + batch], theta[a:a + batch], grad=g, loss=losses[i:i + 1])
                self.adam(g, lr * (lr_final / lr) ** (i / max(total - 1, 1)))
        return losses[:total]

    def predict(self, feat):
        rows = feat.shape[0]
        th = _empty(rows, 3, dtype=torch.float64, device=self.device)
        ws = self.ws(rows)
        _check(lib().pssgp_mlp_predict(_ptr(self.state), _ptr(feat), rows, _ptr(th), _ptr(ws), ws.numel(),
                                       _stream()), "pssgp_mlp_predict")
        return th
