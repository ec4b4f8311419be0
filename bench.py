#!/usr/bin/env python3
"""Benchmark of the parallel state-space GP prediction path on B300.

One step = one pssgp_predict call on the large noisy-sinusoid workload:
merge of 10,000 prediction times into 2^20 sorted training times, Taylor
order-6 RBF state-space model (d = 6), discretisation, parallel Kalman filter
with missing measurements, parallel RTS smoother, gather at the prediction
times and the log marginal likelihood, all FP64.  The metric is merged time
steps per second (N + M = 1,058,576 steps per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rbf6|matern52]

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the path has no cross-series exchange in this configuration);
value = all ranks' steps / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filter+smoother time steps/s at N=2^20,d=6 FP64"
# DRAM bytes per merged step of each kernel, from a one-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels at the
# 2^20 workload itself; a launch's traffic is this x n.  Reset an entry to None
# whenever its kernel changes.
PROFILED_DRAM_BYTES_PER_STEP = {"filter_propagate": 1414.8, "filter_reduce": 478.0, "discretize": 415.4,
                                "smoother_propagate": 682.3}
UNIT = "steps/s"
BATCH_SIM_SEED = 300          # prior simulation of the batched workload (family i: seed + i)
WORKLOADS = {
    "rbf6": dict(kind="rbf", order=6, lengthscale=1.0, variance=1.0, noise=0.01),
    "matern52": dict(kind="matern52", order=0, lengthscale=1.0, variance=1.0, noise=0.01),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rbf6", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--timing-steps", type=int, default=3)
    ap.add_argument("--warps-per-sm", type=int, default=0, help="scan lanes per SM / 32 (0 = library default)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 4,096-series batched measurement")
    ap.add_argument("--streams", type=int, default=8,
                    help="streams (each with its own workspace) that the timed steps alternate over")
    ap.add_argument("--concurrent-warps", type=int, default=2,
                    help="scan lanes per SM / 32 of each prediction while several run on the streams "
                         "(0 = the library default, which targets one prediction at a time)")
    ap.add_argument("--no-fit", action="store_true", help="skip the learned-vs-plain fit and Table-1 measurements")
    ap.add_argument("--no-gradient", action="store_true", help="skip the log-likelihood gradient measurement")
    ap.add_argument("--no-fit-adam", action="store_true", help="skip the Adam fits (about a minute and a half)")
    ap.add_argument("--profile", default="", choices=["", "grad", "batched", "batched_grad", "learn"],
                    help="run one small case 3 times for a profiler and exit (no JSON line)")
    ap.add_argument("--split-series", action="store_true",
                    help="one long series split in contiguous time chunks over the GPUs (strong scaling)")
    ap.add_argument("--n-train", type=int, default=0,
                    help="profile a prefix of the workload with this many training points (0 = full 2^20)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# algorithmic FP64 flop counts per merged step (FMA = 2 flops; a reciprocal,
# square root or comparison counts 1), from the formulas each kernel evaluates
# ---------------------------------------------------------------------------
def flops_discretize(d, kf, kq, companion=True, qrows=True):
    s = d * (d + 1) // 2
    if companion:   # row 0 of F by Horner, rows 1..d-1 by the companion recursion
        f = 2 * d * (kf - 1) + (d - 1) * (1 + 3 * (d - 1))
    else:
        f = 2 * d * d * (kf - 1)
    if companion and qrows:
        # row 0 of Q by Horner and its scaling; row i+1 from row i by the
        # Lyapunov identity: w f_i, 3 flops per inner entry, 1 + 2d for the
        # last column
        q = 2 * d * (kq - 1) + d + (d - 1) * (2 + 2 * d) + 3 * (d - 2) * (d - 1) // 2
    else:
        q = 2 * s * (kq - 1) + s
    return f + q


def diffusion_on_last_state(model):
    """True when W = w e_{d-1} e_{d-1}^T (rows 1..d-1 of Q follow from row 0)."""
    d = model.d
    W = np.ctypeslib.as_array(model.raw.W)[:d * d]
    return bool(W[-1] > 0.0 and np.count_nonzero(W[:-1]) == 0)


def flops_filter_fold(d, observed_frac):
    s = d * (d + 1) // 2
    pred = (2 * d ** 3 - d * d) * 2 + (2 * d * d - d) + 2 * s * d          # F A, F C, F b, (F C) F^T + Q
    upd = 4 + 6 * d + 4 * s + 2 * d * d                                    # S, 1/S, r, w/S, J, eta, K, A, b, C
    return pred + observed_frac * upd


def flops_kf_step(d, observed_frac):
    s = d * (d + 1) // 2
    pred = (2 * d * d - d) + (2 * d ** 3 - d * d) + 2 * s * d              # F x, F P, (F P) F^T + Q
    upd = 6 + 3 * d + 2 * s                                                # S, 1/S, v, K, x, P, log-lik terms
    return pred + observed_frac * upd


def flops_smoother_element(d):
    """E and g from P^- = Lu diag(dd) Lu^T (square-root free; one reciprocal
    per pivot): W = Lu^{-1} T, V = diag(1/dd) W, E^T = Lu^{-T} V,
    g = x - E x^- (the record keeps P_k and P^- instead of L)."""
    ldl = sum(2 * j + 1 + (d - 1 - j) * (2 * j + 1) for j in range(d))
    return ldl + 2 * d * d * (d - 1) + d * d + 2 * d * d


def flops_smoother_fold(d):
    s = d * (d + 1) // 2
    return (2 * d ** 3 - d * d) * 2 + 2 * d * d + 2 * s * d                # E_a E, E_a L, E_a g + g_a, (.)E_a^T + L_a


def flops_rts_step(d):
    """m = E m' + g; P^s = P + E (P^s' - P^-) E^T."""
    s = d * (d + 1) // 2
    return 2 * d * d + s + (2 * d ** 3 - d * d) + 2 * s * d


def flops_adjoint_fold(d, observed_frac):
    """Mean-adjoint chunk product in the filter pass: Pi F^T, Pi[:,0] v/S,
    Pi - Pi[:,0] K^T."""
    return (2 * d ** 3 - d * d) + observed_frac * (2 * d + 2 * d * d)


def flops_adjoint_step(d, observed_frac):
    """One backward step of the covariance adjoint as evaluated: xb = F^T mb,
    F^T M F accumulated row by row (d rows of L F, d x Sym outer updates),
    w = R K, K^T R K, the rank-2 corrections, mb = A xb + e0 v/S."""
    s = d * (d + 1) // 2
    return 2 * d * d + d * (2 * d * d + 2 * s) + observed_frac * (2 * d * d + 2 * d + 2 * d + 8)


def flops_adjoint_terms(d, observed_frac, companion=True):
    """The derivative terms of one step: tr(Mb Q), tr(Mb W), mb^T G m,
    tr(Mb G M) (companion drift: 2d - 1 entries of M Mb), dl/dR."""
    s = d * (d + 1) // 2
    gm = (2 * d - 1) * 2 * d if companion else 2 * d ** 3
    return 4 * s + gm + 4 * d + 8 + observed_frac * 6


def taylor_terms(model, t, lanes, L):
    """Mean Taylor term counts as the device picks them: per warp and per
    in-chunk iteration, from the longest step over the warp's 32 lanes."""
    h = np.diff(t, prepend=t[0])
    h[0] = 0.0
    n = t.size
    hp = np.zeros(lanes * L)
    hp[:n] = h
    hf = np.minimum(hp.reshape(lanes, L).astype(np.float32), np.float32(model.raw.hmax))
    hw = hf.reshape(lanes // 32, 32, L).max(axis=1).ravel()
    thr_f = np.array(model.raw.hthr_f[1:], dtype=np.float32)
    thr_q = np.array(model.raw.hthr_q[1:], dtype=np.float32)
    kf = np.searchsorted(thr_f, hw, side="left") + 1
    kq = np.searchsorted(thr_q, hw, side="left") + 1
    return float(kf.mean()), float(kq.mean())


def lane_plan(n, sms=148, warps_per_sm=4):
    lanes_max = sms * warps_per_sm * 32
    want = (n + 7) // 8
    P0 = min(lanes_max, max(want, 1))
    P0 = (P0 + 127) // 128 * 128
    return P0, (n + P0 - 1) // P0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v: float, world: int, device) -> float:
    """The largest value over all ranks (the slowest rank's time); a no-op on
    one rank.  `device`: where the collective's tensor lives (the GPU for
    NCCL, the CPU for gloo)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of replicas: every rank processes units_per_rank
    in each step; the job's step time is the slowest rank's."""
    return units_per_rank * world / (ms_max * 1e-3)


def fp64_peaks(P, dev, sm_mhz=None):
    """(measured, nominal) FP64 peaks in TFLOP/s: the best launch of the live
    DFMA probe (pssgp_fp64_fma_rate, x2 flops per FMA), and SMs x 128 lanes /
    64 cycles per warp DFMA x 2 flops x the SM clock (the median sampled under
    load, else the maximum)."""
    import torch
    measured = 2 * P.fp64_fma_rate() / 1e12
    props = torch.cuda.get_device_properties(dev)
    mhz = sm_mhz or 2032.0
    nominal = props.multi_processor_count * 128 / 64 * 2 * mhz * 1e6 / 1e12
    return measured, nominal


def roofline_peak_fields(measured, nominal, sm_mhz):
    return {"peak": round(measured, 4), "peak_nominal": round(nominal, 4),
            "peak_source": "measured: best launch of the FP64 DFMA probe on this GPU (pssgp_fp64_fma_rate, "
                           "best of 3 launches at each of 4, 8, 16 warps/SM, x2 flops); nominal: SMs x 128 lanes / "
                           f"64 cycles x 2 flops x {sm_mhz:.0f} MHz"}


CPU_SAMPLE_TRAIN = 1 << 19
REFERENCE_TIMED_S = 120.0     # the reference arm's timed runs stop after about this long


def _oracle_sample_run(wl_params, n_sample_train):
    """One run of the oracle as it stands (merge + sequential KF + RTS +
    log-likelihood) on a prefix sample of the large workload: (merged steps,
    seconds)."""
    import oracle
    import workloads as wl
    from oracle import model as om
    oracle.build()
    s = wl.prefix(wl.sinusoid_large(), n_sample_train)
    o = om.make_model(wl_params["kind"], wl_params["lengthscale"], wl_params["variance"],
                      order=wl_params["order"] or 6)
    t0 = time.perf_counter()
    oracle.predict(o, s.t_train, s.y_train, s.t_test, wl_params["noise"])
    return s.N + s.M, time.perf_counter() - t0, s


def _oracle_sample_desc(s, n, dts, cores, how):
    return (f"first {s.N} training + {s.M} prediction points of the workload ({n} merged steps); {how}: "
            f"{min(dts):.2f} s (all runs {', '.join(f'{x:.2f}' for x in dts)} s); long-double sequential KF + "
            f"RTS, discretisation on {cores} threads")


def cpu_baseline(wl_params, n_sample_train=CPU_SAMPLE_TRAIN, reps=5):
    """The oracle as it stands on the host cores, on a bounded prefix sample of
    the same workload: best of `reps` runs after one warm-up run; steps/s."""
    _oracle_sample_run(wl_params, n_sample_train)            # warm-up (page cache, thread pool)
    dts = []
    for _ in range(reps):
        n, dt, s = _oracle_sample_run(wl_params, n_sample_train)
        dts.append(dt)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n / min(dts), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": _oracle_sample_desc(s, n, dts, cores, f"best of {reps} runs after one warm-up")}


def workload_config(workload, d, n):
    """The `config` object of both arms' JSON lines."""
    return {"workload": f"{workload}: N=2^20 training times U[0,1000] + M=10^4 prediction times, "
                        f"y=sin(0.3t)+0.5sin(1.7t)+N(0,0.1^2), d={d}, l=1, s2=1, R=0.01; "
                        "one pssgp_predict (merge+filter+smoother+gather+loglik) per step",
            "merged_steps": n, "per_rank_replica": True,
            "l2": "workspace traffic ~1 GB per step exceeds the 126 MB L2 (no explicit flush)"}


def run_reference(args, wl_params):
    """The reference arm: the oracle (there is no other implementation of the
    method to install) timed on the host cores on the same bounded sample as
    the cpu_baseline of our arm; `warmup` untimed runs, then `steps` timed
    runs, value = the best timed run (the best-of-runs rule of the CPU
    baseline, so both report the same quantity)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import workloads as wl
    from oracle import model as om
    full = wl.sinusoid_large()
    n_full = int(full.N + full.M)       # merged steps of the timed workload (the sample is a prefix)
    d = om.make_model(wl_params["kind"], wl_params["lengthscale"], wl_params["variance"],
                      order=wl_params["order"] or 6).d
    wdt = 0.0
    for _ in range(max(args.warmup, 1)):
        _, wdt, _ = _oracle_sample_run(wl_params, CPU_SAMPLE_TRAIN)
    # at most about two minutes of timed runs: K runs of the 2^19-point sample
    # when they fit, else as many as fit (the value is the best run either way)
    runs = max(1, min(args.steps, max(3, int(REFERENCE_TIMED_S / max(wdt, 1e-3)))))
    dts = []
    for _ in range(runs):
        n, dt, s = _oracle_sample_run(wl_params, CPU_SAMPLE_TRAIN)
        dts.append(dt)
    v = n / min(dts)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    capped = f" ({args.steps} requested; capped to about {REFERENCE_TIMED_S:.0f} s)" if runs < args.steps else ""
    sample = _oracle_sample_desc(s, n, dts, cores,
                                 f"best of {len(dts)} timed runs{capped} after {max(args.warmup, 1)} warm-up runs")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(dts), "warmup": args.warmup, "ms_per_step": min(dts) * 1e3 * n_full / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, d, n_full),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batched_bench(args, P, wl, dev, barrier, world, rank):
    """Log-likelihood of the 4,096-series batch (lengths log-uniform in
    [1000, 65536], Matern-3/2 / 5/2 mixed, one pssgp_loglik_batched call per
    family), autotuned lane counts, both families replayed as one CUDA graph
    per evaluation; inputs resident in HBM."""
    import torch
    offs, kinds, params = wl.prior_batch_spec(**dict(wl.PRIOR_BATCH, seed=wl.PRIOR_BATCH["seed"] + rank))
    kinds = np.array(kinds)
    B_all = offs.size - 1
    parts = []
    for fi, kind in enumerate(("matern32", "matern52")):
        off, par = wl.subset_spec(offs, params, np.flatnonzero(kinds == kind))
        m = P.build_model(kind, 1.0, 1.0)
        offd = torch.as_tensor(off, device=dev)
        pard = torch.as_tensor(par, device=dev)
        # y drawn from the state-space prior of the series' own model (the
        # library's simulation: Poisson time grid of mean spacing 0.01)
        t, y, st = P.simulate_prior(m, offd, pard, seed=BATCH_SIM_SEED + fi + 10 * rank)
        assert int(st.item()) == 0, "prior simulation status"
        d = dict(kind=kind, m=m, n=t.numel(), B=off.size - 1, off=offd, par=pard, t=t, y=y,
                 mask=torch.ones(t.numel(), dtype=torch.uint8, device=dev))
        d["ws"] = P.workspace(m.d, d["n"], dev)
        d["ll"] = torch.empty(d["B"], dtype=torch.float64, device=dev)
        parts.append(d)
    tuning = {}
    for d in parts:
        w, _ = P.autotune_loglik_batched(d["m"], d["off"], d["par"], d["t"], d["y"], d["mask"], ws=d["ws"],
                                         out=d["ll"])
        tuning[d["kind"]] = {"d": d["m"].d, "warps_per_sm": w}

    def call(d):
        P.loglik_batched(d["m"], d["off"], d["par"], d["t"], d["y"], d["mask"], ws=d["ws"], out=d["ll"])

    for d in parts:
        call(d)
    torch.cuda.synchronize()
    assert all(P.status(d["ws"]) == 0 for d in parts), "device status error (batched)"
    # one family after the other in one graph: as two parallel branches (fork
    # onto a second stream and join) an evaluation took 24.6 ms against 24.0,
    # the lane counts being tuned for the whole GPU
    g = P.Graph()
    with g:
        for d in parts:
            call(d)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        g.launch()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.launch()
    e1.record(stream)
    e1.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    P.timing(1)
    for d in parts:
        call(d)
    torch.cuda.synchronize()
    per = P.timing(2)
    P.timing(0)
    n_all = sum(d["n"] for d in parts)
    pred = batched_predict_bench(args, P, parts, dev, barrier, world)
    return {"workload": "4,096 series, lengths log-uniform [1000, 65536], Matern-3/2 / 5/2 mixed, l log-uniform "
                        "[0.1, 10], s2 = 1, R log-uniform [1e-3, 1e-1], times and y drawn from the SSGP prior of "
                        "each series (Poisson grid of mean spacing 0.01, pssgp_simulate_prior); log-likelihood of "
                        "every series, one pssgp_loglik_batched per family, replayed as one CUDA graph",
            "series": B_all, "steps_total": int(n_all), "ms_per_eval": ms,
            "series_per_s": job_throughput(B_all, world, ms), "steps_per_s": job_throughput(n_all, world, ms),
            "tuning": tuning, "gpu_launches_per_eval": int(sum(c for _, c in per.values())),
            "kernels_ms": {k: round(v[0], 4) for k, v in per.items()},
            "l2": "inputs and workspace ~17 GB per evaluation, far above the 126 MB L2",
            "predict": pred}


def batched_predict_bench(args, P, parts, dev, barrier, world):
    """Posterior predictions of the same 4,096 series in one pssgp_predict_batched
    call per family: a prediction time midway between the training times k and
    k + 1 for every k = 50 mod 100 of each series (1 % of its steps, at least
    one), merged, filtered and smoothed with each series' log-likelihood."""
    import torch
    legs = []
    for d in parts:
        off = d["off"].cpu().numpy()
        idx, uo = [], [0]
        for s in range(off.size - 1):
            a, b = int(off[s]), int(off[s + 1])
            ks = np.arange(a + 50, b - 1, 100) if b - a > 51 else np.array([a] if b - a > 1 else [], dtype=np.int64)
            idx.append(ks)
            uo.append(uo[-1] + ks.size)
        idx_d = torch.as_tensor(np.concatenate(idx).astype(np.int64), device=dev)
        u = 0.5 * (d["t"][idx_d] + d["t"][idx_d + 1])
        uoff = torch.as_tensor(np.array(uo, dtype=np.int64), device=dev)
        ws = P._empty(int(P.lib().pssgp_predict_batched_workspace_size(d["m"].d, d["n"], u.numel(), d["B"])),
                      dtype=torch.uint8, device=dev)
        legs.append((d, u, uoff, ws))

    def call():
        for d, u, uoff, ws in legs:
            P.predict_batched(d["m"], d["off"], uoff, d["par"], d["t"], d["y"], u, ws=ws)

    for _ in range(max(args.warmup, 3)):
        call()
    torch.cuda.synchronize()
    assert all(P.status(ws) == 0 for _, _, _, ws in legs), "device status error (batched prediction)"
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    e1.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    B_all = sum(d["B"] for d, *_ in legs)
    n_all = sum(d["n"] + u.numel() for d, u, *_ in legs)
    return {"what": "posterior mean and variance at 1 % of each series' steps (between training times 50 mod 100) "
                    "and every series' log-likelihood, one pssgp_predict_batched call per family",
            "prediction_times": int(sum(u.numel() for _, u, *_ in legs)), "merged_steps": int(n_all),
            "ms_per_call": ms, "series_per_s": job_throughput(B_all, world, ms),
            "steps_per_s": job_throughput(n_all, world, ms)}


def gradient_bench(args, P, wl, dev, sm_mhz=None):
    """Log-likelihood + gradient (row f2): RBF-6 on the 2^20 training points of
    the large workload (one pssgp_loglik_grad per step, inputs resident), with
    per-kernel times and the roofline of the dominant adjoint kernel."""
    import torch
    s = wl.sinusoid_large()
    m = P.build_model("rbf", 1.0, 1.0)
    t = torch.as_tensor(s.t_train, device=dev)
    y = torch.as_tensor(s.y_train, device=dev)
    mask = torch.ones(t.numel(), dtype=torch.uint8, device=dev)
    ws = P.workspace_grad(m.d, t.numel(), dev)
    wsl = P.workspace(m.d, t.numel(), dev)
    for _ in range(max(args.warmup, 3)):
        P.loglik_grad(m, t, y, mask, 0.01, ws=ws)
    torch.cuda.synchronize()

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    ms_g = timed(lambda: P.loglik_grad(m, t, y, mask, 0.01, ws=ws), args.steps)
    ms_l = timed(lambda: P.loglik(m, t, y, mask, 0.01, ws=wsl), args.steps)
    P.timing(1)
    P.loglik_grad(m, t, y, mask, 0.01, ws=ws)
    torch.cuda.synchronize()
    per = P.timing(2)
    P.timing(0)
    n, d = t.numel(), m.d
    alg = {"adjoint_cov": n * (flops_adjoint_step(d, 1.0) + flops_adjoint_terms(d, 1.0)),
           "adjoint_mean": n * flops_adjoint_step(d, 1.0),
           "filter_propagate": n * (flops_kf_step(d, 1.0) + flops_adjoint_fold(d, 1.0)),
           "filter_reduce": n * flops_filter_fold(d, 1.0)}
    peak, nominal = fp64_peaks(P, dev, sm_mhz)
    dom = max(alg, key=lambda k: per[k][0])
    ach = alg[dom] / (per[dom][0] * 1e-3) / 1e12
    return {"workload": "RBF Taylor-6 (d = 6), the 2^20 training points of the large workload, l = s2 = 1, "
                        "R = 0.01; d loglik / d(log l, log s2, log R)",
            "ms_loglik_grad": round(ms_g, 4), "ms_loglik": round(ms_l, 4), "ratio": round(ms_g / ms_l, 3),
            "steps_per_s": n / (ms_g * 1e-3),
            "kernels_ms": {k: round(v[0], 4) for k, v in per.items()},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": round(ach, 4), "unit": "TFLOP/s",
                         "frac": round(ach / peak, 4), "frac_of_nominal": round(ach / nominal, 4),
                         "ms_per_launch": round(per[dom][0], 4), "algorithmic_flops_per_launch": alg[dom],
                         **roofline_peak_fields(peak, nominal, sm_mhz or 2032.0)}}


def fit_bench(args, P, wl):
    """Learned initialisation (row f3): train the network on 10^6 simulated
    Matern-5/2 prior series of 4,096 steps, then fit 4,096 held-out prior
    series (lengths log-uniform in [4096, 65536]) from the plain default and
    from the network's proposals with the same optimiser; series per second
    of the whole fit (device wall clock) and the share of learned-init fits
    within 1e-3 nats per point of the plain fit's log-likelihood."""
    import torch
    from paper_2102_09964_b300 import learn as L
    m = P.build_model("matern52", 1.0, 1.0)
    offs, params = wl.prior_spec(wl.LEARN_TRAIN["seed"], wl.LEARN_TRAIN["B"], n=wl.LEARN_TRAIN["n"])
    net, train_s, losses = L.train_network(m, offs, params, seed=500, epochs=8)
    ho, hp = wl.prior_spec(**wl.LEARN_HELDOUT)
    t, y = L.heldout_series(m, ho, hp, seed=510)
    out = {"workload": "train: 10^6 Matern-5/2 prior series x 4,096 steps (Poisson grid, mean spacing 0.01), "
                       "l, s2 log-uniform [0.1, 10], R log-uniform [1e-3, 1e-1]; held-out: 4,096 prior series, "
                       "lengths log-uniform [4096, 65536]; plain init l = s2 = R = 1",
           "train_s": round(train_s, 3), "train_loss_final": float(losses[-64:].mean().item()),
           "heldout_steps": int(ho[-1])}
    runs = [("lbfgs", dict(method="lbfgs", patience=3, tol=1e-9, max_iter=500, check_every=1))]
    if not args.no_fit_adam:
        runs.append(("adam", dict(method="adam", patience=10, tol=1e-7, max_iter=2000, check_every=1)))
    for name, kw in runs:
        r = L.compare_fits(net, m, ho, t, y, order="abba", **kw)
        gain = r["plain"]["gpu_s"] - r["learned"]["gpu_s"]
        out[name] = {"plain": r["plain"], "learned": r["learned"], "order": r["order"],
                     "speedup": round(r["plain"]["gpu_s"] / r["learned"]["gpu_s"], 3),
                     "learned_within_1e-3_nats_per_point": r["learned_within_1e-3_nats_per_point"],
                     # the network's training is paid once; one batch of 4,096
                     # series costs train_s + learned gpu_s with the learned start
                     "learned_plus_training_gpu_s_one_batch": round(train_s + r["learned"]["gpu_s"], 3),
                     "break_even_batches": (round(train_s / gain, 2) if gain > 0 else None),
                     "options": kw}
    del t, y
    torch.cuda.empty_cache()
    return out


def table1_bench(P, wl):
    """The paper's learning loop (Sec. 5.2, Table 1) on a shape-only stand-in:
    L-BFGS on the log-likelihood of N = 1200 / 2200 / 3200 monthly points
    (Matern-3/2, start l = s2 = R = 1), milliseconds per function/gradient
    evaluation; then the daily interpolation at 96,000 prediction times."""
    import time
    import torch
    s = wl.sunspot_like()
    out = {"workload": "sunspot-shaped synthetic series (no sunspot data): monthly training times, 96,000 daily "
                       "prediction times, Matern-3/2", "paper_ms_per_eval": {"1200": 39, "2200": 46, "3200": 48},
           "paper_interpolation_s": 0.14, "paper_hardware": "as stated in the paper (context only)"}
    m = P.build_model("matern32", 1.0, 1.0)
    best = None
    for N in (1200, 2200, 3200):
        t = torch.as_tensor(s.t_train[:N], device="cuda")
        y = torch.as_tensor(s.y_train[:N], device="cuda")
        mask = torch.ones(N, dtype=torch.uint8, device="cuda")
        P.fit_batched(m, np.array([0, N]), t, y, mask, np.zeros((1, 3)), method="lbfgs", max_iter=20)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, ll, it, _ = P.fit_batched(m, np.array([0, N]), t, y, mask, np.zeros((1, 3)), method="lbfgs",
                                      patience=3, tol=1e-12, max_iter=500, check_every=10)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ev = int(it[0].item())
        out[f"N{N}"] = {"evaluations": ev, "fit_s": round(dt, 5), "ms_per_eval": round(1e3 * dt / max(ev, 1), 4),
                        "loglik": float(ll[0].item())}
        best = th[0].cpu().numpy()
    ell, s2, R = np.exp(best)
    mf = P.build_model("matern32", float(ell), float(s2))
    tt = torch.as_tensor(s.t_train, device="cuda")
    yy = torch.as_tensor(s.y_train, device="cuda")
    ts = torch.as_tensor(s.t_test, device="cuda")
    ws = P.workspace(mf.d, tt.numel() + ts.numel(), torch.device("cuda"))
    for _ in range(3):
        P.predict(mf, tt, yy, ts, float(R), ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        P.predict(mf, tt, yy, ts, float(R), ws=ws)
    e1.record()
    e1.synchronize()
    out["interpolation_s"] = round(e0.elapsed_time(e1) / 10 / 1e3, 6)
    out["fitted"] = {"lengthscale": float(ell), "variance": float(s2), "noise": float(R)}
    return out


def run_ours(args, wl_params):
    import torch
    import paper_2102_09964_b300 as P
    import workloads as wl
    from paper_2102_09964_b300 import build as B

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    P.lib()
    if args.warps_per_sm:
        P.set_warps_per_sm(args.warps_per_sm)
    dev = torch.device("cuda", torch.cuda.current_device())
    s = wl.sinusoid_large(seed=2 + rank)
    if args.n_train:
        s = wl.prefix(s, args.n_train)
    N, M = s.N, s.M
    n = N + M
    m = P.build_model(wl_params["kind"], wl_params["lengthscale"], wl_params["variance"],
                      order=wl_params["order"] or 6)
    R = wl_params["noise"]
    tt = torch.as_tensor(s.t_train, dtype=torch.float64, device=dev)
    yy = torch.as_tensor(s.y_train, dtype=torch.float64, device=dev)
    ts = torch.as_tensor(s.t_test, dtype=torch.float64, device=dev)
    wsb = P.workspace(m.d, n, dev)
    out = (torch.empty(M, dtype=torch.float64, device=dev), torch.empty(M, dtype=torch.float64, device=dev),
           torch.empty(1, dtype=torch.float64, device=dev))
    stream = torch.cuda.current_stream()

    def step():
        P.predict(m, tt, yy, ts, R, ws=wsb, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert P.status(wsb) == 0, "device status error"

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # --- device-timed region (inputs resident in HBM) ---
    # one stream first at the library's default tuning (reported as
    # ms_per_step_one_stream: the latency of one prediction), then the timed
    # value: steps alternate between --streams streams with a workspace each,
    # each prediction on --concurrent-warps warps per SM (fewer, longer lane
    # chunks: less scan overhead per step, while the predictions in flight
    # together fill the SMs; one step's low-occupancy scan rounds also
    # overlap the other steps' kernels)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    ms_one = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)

    ns = max(1, args.streams)
    w_default = P.tune_get(m.d)
    w_conc = args.concurrent_warps or w_default
    P.tune_set(m.d, w_conc)
    dstreams = [torch.cuda.Stream() for _ in range(ns)]
    wsbs = [wsb] + [P.workspace(m.d, n, dev) for _ in range(ns - 1)]
    outs = [out] + [tuple(torch.empty_like(o) for o in out) for _ in range(ns - 1)]

    def dstep(i):
        j = i % ns
        with torch.cuda.stream(dstreams[j]):
            P.predict(m, tt, yy, ts, R, ws=wsbs[j], out=outs[j])

    for i in range(max(args.warmup, 3) + ns - 1):
        dstep(i)
    torch.cuda.synchronize()
    assert all(P.status(w) == 0 for w in wsbs), "device status error"
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for st in dstreams:
        st.wait_stream(stream)
    for i in range(args.steps):
        dstep(i)
    for st in dstreams:
        stream.wait_stream(st)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(n, world, ms)
    del wsbs[1:]

    # --- end to end through the C ABI from pinned host buffers ---
    # pssgp_predict_host: every step copies its inputs host -> device and its
    # results device -> host inside the call; --streams streams with a workspace each
    # let one step's copies overlap the other's kernels
    h_tt = torch.as_tensor(s.t_train, dtype=torch.float64).pin_memory()
    h_yy = torch.as_tensor(s.y_train, dtype=torch.float64).pin_memory()
    h_ts = torch.as_tensor(s.t_test, dtype=torch.float64).pin_memory()
    streams = [torch.cuda.Stream() for _ in range(ns)]
    houts = [(torch.empty(M, dtype=torch.float64).pin_memory(), torch.empty(M, dtype=torch.float64).pin_memory(),
              torch.empty(1, dtype=torch.float64).pin_memory()) for _ in streams]
    hws = [None] * ns

    def e2e_step(i):
        j = i % ns
        hws[j] = P.predict_host(m, h_tt, h_yy, h_ts, R, houts[j], ws=hws[j], stream=streams[j])

    for i in range(2 * ns):
        e2e_step(i)
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for st in streams:
        st.wait_stream(stream)
    for i in range(args.steps):
        e2e_step(i)
    for st in streams:
        stream.wait_stream(st)
    f1.record(stream)
    f1.synchronize()
    ms_e2e = f0.elapsed_time(f1) / args.steps
    ms_e2e = max_over_ranks(ms_e2e, world, dev)
    e2e = {"value": job_throughput(n, world, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": int((2 * N + M) * 8), "d2h_bytes_per_step": int((2 * M + 1) * 8)}

    # launches per step at the tuning of the timed region
    P.timing(1)
    step()
    torch.cuda.synchronize()
    gpu_launches = sum(c for _, c in P.timing(2).values()) * args.steps
    P.timing(0)
    P.tune_set(m.d, w_default)

    # --- per-kernel times (events around each launch) for the roofline, at
    # the default tuning (one prediction on the whole GPU) ---
    P.timing(1)
    for _ in range(args.timing_steps):
        step()
    torch.cuda.synchronize()
    per = P.timing(2)
    P.timing(0)
    sm_mhz = clocks.get("sm_mhz") if isinstance(clocks, dict) else None
    peak_tflops, nominal_tflops = fp64_peaks(P, dev, sm_mhz)

    t_merged = np.sort(np.concatenate([s.t_train, s.t_test]), kind="stable")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    lanes, L = lane_plan(n, sms, w_default)
    kf, kq = taylor_terms(m, t_merged, lanes, L)
    d = m.d
    obs = N / n
    alg = {
        "discretize": n * flops_discretize(d, kf, kq, bool(m.raw.companion), diffusion_on_last_state(m)),
        "filter_reduce": n * flops_filter_fold(d, obs),
        # the smoother chunk aggregate is formed once per lane (not per step)
        "filter_propagate": n * (flops_kf_step(d, obs) + flops_smoother_element(d)),
        "smoother_propagate": n * flops_rts_step(d),
    }
    ts = max(args.timing_steps, 1)
    kernels = {}
    for name, (tot, cnt) in per.items():
        kernels[name] = {"ms_per_step": round(tot / ts, 4), "launches_per_step": cnt // ts,
                         "ms_per_launch": round(tot / cnt, 4), "share": None}
    tot_all = sum(v["ms_per_step"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = round(v["ms_per_step"] / tot_all, 4)
    dom = max((k for k in alg if k in kernels), key=lambda k: kernels[k]["ms_per_step"])
    achieved = alg[dom] / (kernels[dom]["ms_per_launch"] * 1e-3) / 1e12
    tb = PROFILED_DRAM_BYTES_PER_STEP.get(dom) if args.workload == "rbf6" else None
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tflops, 4), "frac_of_nominal": round(achieved / nominal_tflops, 4),
                "traffic": (tb * n if tb else None), "kernel": dom,
                "ms_per_launch": kernels[dom]["ms_per_launch"], "algorithmic_flops_per_launch": alg[dom],
                **roofline_peak_fields(peak_tflops, nominal_tflops, sm_mhz or 2032.0),
                "taylor_terms": {"F": round(kf, 2), "Q": round(kq, 2)}}
    whole = sum(alg.values()) / (ms * 1e-3) / 1e12

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_one_stream": round(ms_one, 4),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, d, n),
            "concurrency": f"value and e2e: {ns} predictions in flight on {ns} streams, each on "
                           f"{w_conc} warps per SM ({lane_plan(n, sms, w_conc)[0]} lane chunks); "
                           f"ms_per_step_one_stream and roofline: one prediction at a time on "
                           f"{w_default} warps per SM ({lane_plan(n, sms, w_default)[0]} lane chunks)",
            "e2e": e2e, "gpu_launches": int(gpu_launches), "clocks": clocks, "roofline": roofline,
            "whole_path_tflops": round(whole, 4), "whole_path_frac": round(whole / peak_tflops, 4),
            "kernels": kernels}
    if not args.no_batched:
        line["batched"] = batched_bench(args, P, wl, dev, barrier, world, rank)
    if not args.no_gradient:
        line["gradient"] = gradient_bench(args, P, wl, dev, sm_mhz)
    if not args.no_fit:
        line["fit"] = fit_bench(args, P, wl)
        line["table1"] = table1_bench(P, wl)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl_params)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def profile_case(args):
    """Small cases for ncu captures (inputs larger than L2, a few GB at most):
    grad: log-likelihood + gradient of RBF-6 on 2^18 training points;
    batched / batched_grad: log-likelihood (+ gradient) of 256 Matern-5/2
    series of the batched workload's length range; learn: prior simulation and
    features of 16,384 series x 4,096 steps and 8 training steps."""
    import torch
    import paper_2102_09964_b300 as P
    import workloads as wl
    from paper_2102_09964_b300 import build as B
    torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", 0)
    if args.profile == "grad":
        s = wl.prefix(wl.sinusoid_large(), 1 << 18)
        m = P.build_model("rbf", 1.0, 1.0)
        t = torch.as_tensor(s.t_train, device=dev)
        y = torch.as_tensor(s.y_train, device=dev)
        mask = torch.ones(t.numel(), dtype=torch.uint8, device=dev)
        ws = P.workspace_grad(m.d, t.numel(), dev)
        for _ in range(3):
            P.loglik_grad(m, t, y, mask, 0.01, ws=ws)
    elif args.profile in ("batched", "batched_grad"):
        bt = wl.series_batch(seed=3, B=256)
        m = P.build_model("matern52", 1.0, 1.0)
        a = (torch.as_tensor(bt.offsets, device=dev), torch.as_tensor(bt.params(), device=dev),
             torch.as_tensor(bt.t, device=dev), torch.as_tensor(bt.y, device=dev),
             torch.ones(bt.t.size, dtype=torch.uint8, device=dev))
        ws = (P.workspace_grad if args.profile == "batched_grad" else P.workspace)(m.d, bt.t.size, dev)
        for _ in range(3):
            if args.profile == "batched":
                P.loglik_batched(m, *a, ws=ws)
            else:
                P.loglik_grad_batched(m, *a, ws=ws)
    else:
        from paper_2102_09964_b300 import learn as L
        m = P.build_model("matern52", 1.0, 1.0)
        offs, params = wl.prior_spec(50, 16_384, n=4096)
        for _ in range(3):
            feat = L.prior_features(m, offs, params, seed=500)
        net = P.MLP(dev)
        th = torch.as_tensor(np.log(params), device=dev)
        net.init(1, feat, th)
        net.train(feat, th, epochs=1, batch=2048)
    torch.cuda.synchronize()
    return 0


def run_split(args, wl_params):
    """One long series split in G contiguous time chunks, one per rank
    (strong scaling: the whole job is one 2^20 + 10^4-step workload).  Each
    step, on every rank: pssgp_merge of the training and prediction times in
    its time range [1000 r / G, 1000 (r+1) / G), then the exchange of
    paper_2102_09964_b300.split (filter reduce, all-gather, filter finish,
    smoother reduce, all-gather, log-likelihood all-reduce, smoother finish);
    outputs: f-mean and f-var at every merged step and the total
    log-likelihood.  Inputs resident in HBM."""
    import torch
    import paper_2102_09964_b300 as P
    import workloads as wl
    from paper_2102_09964_b300 import build as B
    from paper_2102_09964_b300 import split as SP

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    P.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    s = wl.sinusoid_large()                       # the same series on every rank
    lo, hi = 1000.0 * rank / world, 1000.0 * (rank + 1) / world
    sel = lambda t: (t >= lo) & ((t < hi) if rank + 1 < world else (t <= hi))
    a, b = sel(s.t_train), sel(s.t_test)
    tt = torch.as_tensor(s.t_train[a], dtype=torch.float64, device=dev)
    yy = torch.as_tensor(s.y_train[a], dtype=torch.float64, device=dev)
    ts = torch.as_tensor(s.t_test[b], dtype=torch.float64, device=dev)
    n_rank = tt.numel() + ts.numel()
    n_total = s.N + s.M
    m = P.build_model(wl_params["kind"], wl_params["lengthscale"], wl_params["variance"],
                      order=wl_params["order"] or 6)
    R = wl_params["noise"]
    ws = P.workspace(m.d, n_rank, dev)
    mws = P._empty(256, dtype=torch.uint8, device=dev)

    def step():
        t, y, mask, _, _ = P.merge(tt, yy, ts, ws=mws)
        gen = SP.chunk_protocol(SP.LibraryChunk(m, t, y, mask, R, ws=ws), rank, world)
        return SP.run_distributed(gen) if world > 1 else SP.run_lockstep([gen])[0]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        fm, fv, ll = step()
    torch.cuda.synchronize()
    assert P.status(ws) == 0 and P.status(mws) == 0, "device status error"
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    P.timing(1)
    step()
    torch.cuda.synchronize()
    per = P.timing(2)
    P.timing(0)
    # + the kernels the timing slots do not cover: two aggregate packs, and a
    # fold and an apply per exchange direction that has other chunks
    launches = sum(c for _, c in per.values()) + 2 + 2 * (rank > 0) + 2 * (rank + 1 < world)

    # the gradient of the log-likelihood over the same split (training times
    # only, grad_protocol), timed after the prediction steps
    gws = P.workspace_grad(m.d, tt.numel(), dev)
    gmask = torch.ones(tt.numel(), dtype=torch.uint8, device=dev)

    def gstep():
        gen = SP.grad_protocol(SP.LibraryChunk(m, tt, yy, gmask, R, ws=gws, grad=True), rank, world)
        return SP.run_distributed(gen) if world > 1 else SP.run_lockstep([gen])[0]

    for _ in range(max(args.warmup, 3)):
        gstep()
    torch.cuda.synchronize()
    assert P.status(gws) == 0, "device status error (split gradient)"
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        gstep()
    g1.record(stream)
    g1.synchronize()
    barrier()
    gms = max_over_ranks(g0.elapsed_time(g1) / args.steps, world, dev)
    line = {"metric": METRIC, "value": n_total / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: one series of 2^20 training + 10^4 prediction times split in "
                                   f"{world} contiguous time chunks (one per GPU); merge + filter + smoother + "
                                   "log-likelihood, f-mean and f-var at every merged step",
                       "merged_steps_total": int(n_total), "merged_steps_this_rank": int(n_rank),
                       "l2": "workspace traffic ~1 GB per step exceeds the 126 MB L2 (no explicit flush)"},
            "gpu_launches": int(launches * args.steps), "clocks": clocks,
            "kernels_ms": {k: round(v[0], 4) for k, v in per.items()},
            "gradient": {"what": "log-likelihood and its gradient (log lengthscale, log variance, log noise) of "
                                 "the 2^20 training steps over the same split (three all-gathers, one all-reduce)",
                         "ms_per_eval": round(gms, 4), "steps_per_s": s.N / (gms * 1e-3)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.profile:
        return profile_case(args)
    wl_params = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl_params)
    if args.split_series:
        return run_split(args, wl_params)
    return run_ours(args, wl_params)


if __name__ == "__main__":
    sys.exit(main())
