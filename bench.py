"""Benchmark of the reduced QMC matrix-vector product on one GB300 (or N replicas).

A step is one pass of the whole hot path over the Gaussian-expectation workload
(reduced rank-1 lattice, b=2, m=16 -> N=65536, s=tau=512, w_j=min(floor(log2(j+1)),10),
one random shift, inverse-normal transform, A=L^T of the exp(-|t_i-t_j|/0.1) covariance,
f=max(mean_t exp(0.2 y_t)-1,0)): point generation, transform, coarse block products, the
fused periodic broadcast-accumulate with f and the mean, and the folded adjoint dQ/dA.
Metric: x_k^T A outputs per second, N*tau*R / step time.  The headline tier is the split
tier (bf16x6 tensor-core coarse block products, FP32 elsewhere); the FP32 and plain-bf16
tiers are timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision split|fp32|bf16]
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
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "x_k^T A products/sec (N*tau/s) vs dense X*A on same GB300, at stated rel. error"
L2_FLUSH_BYTES = 512 << 20        # > 129 MB L2
SM_COUNT = 152
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel on this workload, from the
# ncu captures summarised under profiles/ (cold cache); a kernel missing here has changed since
# its counters were taken and reports traffic null
TRAFFIC_BYTES = {"k_fine_bwd_s4": 10012928, "k_fine_fwd_s4": 9484544, "k_coarse_grad_tc": 17909248,
                 "k_coarse_fwd_tc": 2355712}
TIERS = ("split", "fp32", "bf16")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=list(TIERS), default="split")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense X*A comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--workload", choices=["c2", "c3", "c5", "basket"], default="c2",
                    help="c2: the contract line (default); c3, c5, basket: a timing line for a larger "
                         "workload (graph-replayed step, per-kernel trace), not the contract line")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed (replicas)

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        return dist, rank, world
    return None, 0, 1


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- workload

def workload():
    from paper_2305_11645_gb300 import inputs as I
    return I.c2(dtype=np.float32)


def band_of(p):
    """Fine band the library's planner picks for this rule (JF levels expanded per root)."""
    m = p.m
    tau_I = [int(np.sum(np.minimum(p.w, m) == I)) for I in range(m + 1)]
    if m >= 4 and all(tau_I[I] <= k for I, k in enumerate([1, 2, 4, 8])):
        jf = 4
    elif m >= 1 and tau_I[0] <= 16:
        jf = 1
    else:
        jf = 0
    chain = [I for I in range(jf, m + 1) if tau_I[I] > 0]
    return jf, tau_I, chain


H_OPS = {1: (0, 0), 2: (1, 1), 3: (1, 1), 4: (1, 0), 5: (3, 1), 6: (1, 1)}   # (fp32 ops, mufu ops) per h(y)
# MUFU (ex2, sin, cos, rcp) lanes per SM per clock: ncu's peak for the XU pipe is one warp
# instruction per 4 cycles per SM sub-partition (measured: an ex2 loop reaches 27.6 per clock)
MUFU_LANES = 32


def fine_work(p, name):
    """Algorithmic work of one launch of the fine-band (S4) kernel, counted per output of all
    shifts: the tree's multiply-adds sum_{I<4} tau_I 2^-I (4 for a full band), h(y) and the row
    accumulation (forward); the recomputed tree, G = coef h'(y) (h' and a multiply), the fold
    (one add per output amortised) and the gradient multiply-adds (adjoint).  Returns (FP32
    pipe operations, an FMA counted once, MUFU operations)."""
    jf, tau_I, _ = band_of(p)
    outs = p.N * p.tau * p.R_eff
    fma = sum(tau_I[I] / 2.0 ** I for I in range(jf))
    fp_h, mufu_h = H_OPS[p.f_kind]
    per = (fma + fp_h + 1) if "fwd" in name else (2 * fma + fp_h + 2)
    return outs * per, outs * mufu_h


def coarse_mma_flops(p, pieces):
    """MMA flops of a coarse block-product launch (forward X_I A_I or adjoint X_I^T F_I, the
    same contraction sizes): 2 n_I tau tau_I per level I >= 4 (n_I = 2^(m-I) distinct rows),
    times the piece products (6 in the split tier, 1 in the bf16 tier)."""
    jf, tau_I, chain = band_of(p)
    np_ = 6 if pieces == 3 else 1
    return sum(2.0 * 2 ** (p.m - I) * p.tau * tau_I[I] for I in chain if I < p.m + 1) * p.R_eff * np_


def tensor_roofline(flops, seconds, peak_tflops):
    return {"bound": "tensor", "achieved": flops / seconds / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": flops / seconds / 1e12 / peak_tflops}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        return mp, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_roofline(fp32_ops, mufu_ops, seconds, clock_mhz):
    """FP32 pipe: 128 FMA lanes/SM/clk (the paired FFMA2 does two per lane in two cycles); MUFU:
    MUFU_LANES/SM/clk.  The bound is the pipe with the larger time at full rate."""
    clk = clock_mhz * 1e6
    p_fp32 = SM_COUNT * 128 * clk
    p_mufu = SM_COUNT * MUFU_LANES * clk
    t_fp32, t_mufu = fp32_ops / p_fp32, mufu_ops / p_mufu
    if t_mufu > t_fp32:
        return {"bound": "alu", "pipe": "mufu", "achieved": mufu_ops / seconds / 1e9, "peak": p_mufu / 1e9,
                "unit": "Gop/s", "frac": t_mufu / seconds}
    return {"bound": "alu", "pipe": "fp32", "achieved": fp32_ops / seconds / 1e9, "peak": p_fp32 / 1e9,
            "unit": "Gop/s", "frac": t_fp32 / seconds}


# ----------------------------------------------------------------------------- our arm

def run_ours(args, dist, rank, world):
    from paper_2305_11645_gb300 import _lib as L
    from paper_2305_11645_gb300 import api
    from paper_2305_11645_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(dist)
    dev = torch.device("cuda", torch.cuda.current_device())
    p = workload()
    rule = api.Rule.from_problem(p)
    f = api.Integrand(p.f_kind, p.f_params)
    A = torch.from_numpy(p.A).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the step as a user runs it repeatedly: one CUDA graph of the forward and backward launches
    prec = args.precision
    integ = api.Integrator(rule, A, f, backward=True, graph=True, precision=prec)
    eager = api.Integrator(rule, A, f, backward=True, graph=False, precision=prec)
    others = {t: api.Integrator(rule, A, f, backward=True, graph=True, precision=t) for t in TIERS if t != prec}
    step = integ.run

    for _ in range(args.warmup):
        step()
        eager.run()
        for o in others.values():
            o.run()
    torch.cuda.synchronize()

    def timed(fn, trace=False, prequeue=False):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(dist)
        torch.cuda.synchronize()
        if trace:
            L.trace_enable(True)
        for a, b in evs:
            flush.zero_()
            if prequeue:
                torch.cuda._sleep(3_000_000)    # the host queues the whole step before the GPU reaches it
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        kern = None
        if trace:
            L.trace_enable(False)
            kern = L.trace_collect()
        return [a.elapsed_time(b) for a, b in evs], kern

    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    times, _ = timed(step)
    clock_info = clocks.stop()
    ms = statistics.mean(times)
    ms_max = max_over_ranks(dist, ms)
    outputs = p.N * p.tau * p.R_eff
    value = world * outputs / (ms_max / 1e3)
    eager_ms = statistics.mean(timed(eager.run)[0])
    tier_ms = {prec: ms}
    for t, o in others.items():
        tier_ms[t] = statistics.mean(timed(o.run)[0])

    # the same steps launched eagerly with the library's per-kernel events, the stream pre-queued
    # so each pair of events brackets device time only (roofline of the dominant kernel)
    ttimes, kern = timed(eager.run, trace=True, prequeue=True)
    launches = sum(c for c, _ in kern.values())
    top = max(kern.items(), key=lambda kv: kv[1][1])
    mp, peak_src = peaks()
    clk = clock_info["sm_mhz"] or mp.get("sm_max_mhz", 2070.0)
    name, (cnt, tot) = top
    per_launch = tot / cnt / 1e3
    if name.endswith("_tc"):
        fl = coarse_mma_flops(p, 3 if prec == "split" else 1)
        roof = tensor_roofline(fl, per_launch, mp["bf16_tflops"])
        roof["peak_source"] = f"{peak_src} dense bf16 burst peak (MEASURED_PEAKS.json bf16_tflops)"
        roof["work"] = {"mma_flops": fl}
    else:
        w32, wmu = fine_work(p, name)
        roof = alu_roofline(w32, wmu, per_launch, clk)
        roof["peak_source"] = (f"derived: {SM_COUNT} SMs x pipe lanes (FP32 128, MUFU {MUFU_LANES}) x median SM "
                               f"clock {clk:.0f} MHz sampled during the timed region")
        roof["work"] = {"fp32_ops": w32, "mufu_ops": wmu}
    roof.update({"kernel": name, "launch_ms": per_launch * 1e3, "traffic": TRAFFIC_BYTES.get(name)})
    kernels = {k: {"launches": c, "ms_per_step": t / args.steps} for k, (c, t) in sorted(kern.items())}

    # the materialised product P = X A of the same workload and tier (qmc_reduced_matmul): its
    # band kernel is bound by the output writes, 4 bytes per output (the root values and the
    # point table it reads are under 5 % of that)
    mws = torch.empty(max(api.workspace_size(L.QMC_OP_REDUCED_MATMUL, [rule], [p.tau], None,
                                             api._precision(A, prec)), 256), dtype=torch.uint8, device=dev)

    def materialize():
        api.reduced_matmul(rule, A, ws=mws, precision=prec)

    for _ in range(3):
        materialize()
    mat_ms = statistics.mean(timed(materialize)[0])
    _, mkern = timed(materialize, trace=True, prequeue=True)
    out_bytes = outputs * 4
    materialized = {"op": "qmc_reduced_matmul (P = X A, R x N x tau float32)", "ms_per_call": mat_ms,
                    "value": outputs / (mat_ms / 1e3), "unit": "outputs/s",
                    "kernels": {k: {"launches": c, "ms_per_call": t / args.steps} for k, (c, t) in sorted(mkern.items())}}
    band = "k_fine_mat_s4" if "k_fine_mat_s4" in mkern else "k_fine_fwd_materialize"
    if band in mkern:
        cnt, tot = mkern[band]
        sec = tot / cnt / 1e3
        materialized["roofline"] = {"bound": "hbm", "kernel": band, "achieved": out_bytes / sec / 1e9,
                                    "peak": mp["hbm_gbs"], "unit": "GB/s", "frac": out_bytes / sec / 1e9 / mp["hbm_gbs"],
                                    "bytes_per_launch": out_bytes, "launch_ms": sec * 1e3, "traffic": None,
                                    "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    del mws

    # end to end through the public API with host buffers: H2D of A, D2H of the estimates and dQ/dA
    A_host = torch.from_numpy(p.A).pin_memory()
    est_host = torch.empty(p.R_eff + 1, dtype=torch.float64).pin_memory()
    grad_host = torch.empty(p.A.shape, dtype=torch.float32).pin_memory()

    def e2e_step():
        integ.A.copy_(A_host, non_blocking=True)
        est, grad = integ.run()
        est_host.copy_(est, non_blocking=True)
        grad_host.copy_(grad, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    for _ in range(2):
        e2e_step()
    etimes, _ = timed(e2e_step)
    e_ms = max_over_ranks(dist, statistics.mean(etimes))
    e2e = {"value": world * outputs / (e_ms / 1e3), "unit": "outputs/s", "ms_per_step": e_ms,
           "h2d_bytes_per_step": int(A_host.numel() * 4),
           "d2h_bytes_per_step": int(est_host.numel() * 8 + grad_host.numel() * 4)}

    result = {"metric": METRIC, "value": value, "unit": "outputs/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": {"split": "bf16x6+f32", "fp32": "f32", "bf16": "bf16+f32"}[prec],
              "data": "synthetic",
              "config": {"workload": "c2 Gaussian expectation: reduced rank-1 lattice b=2 m=16 (N=65536), "
                                     "s=tau=512, w_j=min(floor(log2(j+1)),10), 1 odd 32-bit shift, inverse-normal "
                                     "transform, A=L^T (exp covariance), f=max(mean exp(0.2y)-1,0)",
                         "N": p.N, "s": p.s, "tau": p.tau, "R": p.R_eff, "precision": prec,
                         "step": "qmc_integrate + qmc_integrate_backward (reuse forward workspace), "
                                 "replayed as one CUDA graph (api.Integrator)",
                         "l2": "flushed before every timed step (512 MiB write, untimed)",
                         "parallelism": "replicas" if world > 1 else "single"},
              "eager_ms_per_step": eager_ms,
              "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clock_info,
              "kernels": kernels, "materialized": materialized, "peaks": peak_src}

    est, grad = step()
    torch.cuda.synchronize()
    if rank == 0:
        result["accuracy"] = accuracy(p, est, grad, args, prec)
        tiers = {}
        for t in TIERS:
            e_t, g_t = (est, grad) if t == prec else others[t].run()
            torch.cuda.synchronize()
            tiers[t] = {"ms_per_step": tier_ms[t], "value": outputs / (tier_ms[t] / 1e3),
                        **accuracy(p, e_t, g_t, args, t)}
        result["tiers"] = tiers
        if not args.no_dense:
            result["dense_xa"] = dense_baseline(p, rule, A, args, flush, stream)
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(p, budget_s=12.0)
    return result


_ORACLE_CACHE = {}


def oracle_full(p):
    if "full" not in _ORACLE_CACHE:
        from oracle import qmc_oracle as O
        Q, mean = O.estimate(p)
        _ORACLE_CACHE["full"] = (mean, O.grad(p))
    return _ORACLE_CACHE["full"]


# stated tolerances on the estimate (relative) and the gradient (max-norm relative) per tier
TOLERANCE = {"split": (1e-6, 1e-6), "fp32": (2e-5, 2e-5), "bf16": (2e-3, 2e-2)}


def accuracy(p, est, grad, args, tier):
    mean, G = oracle_full(p)
    e = est.cpu().numpy()[-1]
    g = grad.double().cpu().numpy()
    return {"estimate": float(e), "oracle_estimate": float(mean), "estimate_rel_err": float(abs(e - mean) / abs(mean)),
            "grad_rel_err": float(np.max(np.abs(g - G)) / np.max(np.abs(G))),
            "tolerance": {"estimate": TOLERANCE[tier][0], "grad": TOLERANCE[tier][1]}}


def dense_baseline(p, rule, A, args, flush, stream):
    """Dense X*A on the same GPU: X materialised once by gen_points (untimed), then per step
    Y = X A (torch.matmul), f, the mean, and dQ/dA = X^T G -- FP32 (TF32 off) and BF16."""
    from paper_2305_11645_gb300 import api
    x32 = api.gen_points(rule, "full", 0, device=A.device).to(torch.int64) & 0xFFFFFFFF
    X = x32.double().mul_(2.0 ** -32)
    X = torch.special.ndtri(X).float()
    c, K = p.f_params[0], p.f_params[1]
    out = {}
    mean, G_or = oracle_full(p)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        Xd, Ad = X.to(dt), A.to(dt)

        def step():
            Y = Xd @ Ad
            E = torch.exp(c * Y.float())
            m_ = E.mean(dim=1)
            fval = torch.clamp(m_ - K, min=0.0)
            est = fval.double().mean()
            Gm = (c * E / p.tau) * (m_ > K).float()[:, None] / p.N
            grad = Xd.t() @ Gm.to(dt)
            return est, grad

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            est, grad = step()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.mean(ts)
        g = grad.double().cpu().numpy()
        out[name] = {"value": p.N * p.tau / (ms / 1e3), "unit": "outputs/s", "ms_per_step": ms,
                     "estimate_rel_err": float(abs(est.item() - mean) / abs(mean)),
                     "grad_rel_err": float(np.max(np.abs(g - G_or)) / np.max(np.abs(G_or)))}
    torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def cpu_baseline(p, budget_s: float = 12.0, rows: int = None):
    """The oracle as it stands (numpy FP64: points from the unreduced definition, inverse normal,
    dense X A, f, X^T grad f) on a bounded sample of the workload's rows."""
    from oracle import qmc_oracle as O
    rows = rows or 4096
    ks = np.arange(rows, dtype=np.int64)
    t0 = time.perf_counter()
    done = 0
    while True:
        X = O.points(p, 0, ks + done % p.N)
        Y = O.product(X, p.A)
        O.integrand(p.f_kind, p.f_params, Y).sum()
        X.T @ O.integrand_grad(p.f_kind, p.f_params, Y)
        done += rows
        el = time.perf_counter() - t0
        if el >= budget_s or done >= p.N:
            break
    cores = len(os.sched_getaffinity(0))
    return {"value": done * p.tau / el, "unit": "outputs/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of {p.N} rows of the workload (shift 0), forward estimate terms and X^T grad f, "
                      f"numpy FP64 (BLAS matmul may use up to {cores} threads, the rest one thread), {el:.1f} s"}


# ----------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return None
    p = workload()
    rows = 2048
    from oracle import qmc_oracle as O

    def step(i):
        ks = (np.arange(rows, dtype=np.int64) + i * rows) % p.N
        X = O.points(p, 0, ks)
        Y = O.product(X, p.A)
        O.integrand(p.f_kind, p.f_params, Y).sum()
        X.T @ O.integrand_grad(p.f_kind, p.f_params, Y)

    for i in range(args.warmup):
        step(i)
    ts = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + i)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(ts)
    value = rows * p.tau / (ms / 1e3)
    cores = len(os.sched_getaffinity(0))
    sample = f"{rows} rows of the workload per step (shift 0), numpy FP64 oracle: forward terms and X^T grad f"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "outputs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c2 Gaussian expectation (see ours); bounded row sample per step",
                       "N": p.N, "s": p.s, "tau": p.tau, "R": p.R_eff, "rows_per_step": rows},
            "cpu_baseline": {"value": value, "unit": "outputs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "outputs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_workload(args):
    """A timing line for one of the larger workloads (the c2 contract line is run_ours):
    the graph-replayed step with L2 flushed before each step (median over the steps), and the
    library's per-kernel trace of eager steps."""
    import torch
    from paper_2305_11645_gb300 import _lib as L
    from paper_2305_11645_gb300 import api
    from paper_2305_11645_gb300 import inputs as I
    prec = args.precision
    if args.workload == "c3":
        p, backward, desc = I.c3(), False, ("c3 reduced periodic digital net b=2 m=20 (N=1048576), s=tau=1024, "
                                            "w_j=min(floor(log2(j+1)),12), 16 XOR shifts, f=exp(-|y|^2/(2 tau)), estimate")
    elif args.workload == "c5":
        p, backward, desc = I.c5(), True, ("c5 reduced rank-1 lattice b=2 m=20 (N=1048576), s=tau=1024, "
                                           "w_j=min(floor(log2(j+1)),12), 8 shifts, f=log sum exp(y), estimate + adjoint")
    else:
        m, s = 25, 10
        sig, rho, S0, K = 0.4, 0.2, 100.0, 110.0
        Sig = np.diag([sig] * s) + np.diag([rho] * (s - 1), 1) + np.diag([rho] * (s - 1), -1)
        A = np.linalg.cholesky(Sig).T.astype(np.float32)
        w = np.array([min(int(math.floor(math.log2(j))), m) for j in range(1, s + 1)], dtype=np.uint32)
        y = I.mc_samples(I.rng(6, I.P_MISC), m, w, 1, force_odd=True)
        p = I.Problem(I.REDUCED_MC, m, w, A, y=y, transform=I.T_INV_NORMAL, f_kind=I.F_CALL_MEAN_EXP,
                      f_params=(1.0, K / S0 * math.exp(sig / 2), 0, 0))
        backward, desc = False, ("basket option by reduced Monte Carlo: m=25 (N=33554432), s=tau=10, "
                                 "w_j=floor(log2 j) (1-based), tridiagonal Sigma (0.4, 0.2), K=110, one replica")
    dev = torch.device("cuda", 0)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(dev)
    f = api.Integrand(p.f_kind, p.f_params)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    it = api.Integrator(rule, A, f, backward=backward, graph=True, precision=prec)
    for _ in range(args.warmup):
        it.run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        it.run()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    eager = api.Integrator(rule, A, f, backward=backward, graph=False, precision=prec)
    eager.run()
    torch.cuda.synchronize()
    L.trace_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(3_000_000)        # the host queues the whole step before the GPU reaches it
        eager.run()
    torch.cuda.synchronize()
    kern = L.trace_collect()
    L.trace_enable(False)
    L.device_status()
    ms = float(np.median(ts))
    outputs = p.N * p.tau * p.R_eff
    return {"workload": args.workload, "description": desc, "metric": METRIC, "value": outputs / (ms / 1e3),
            "unit": "outputs/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "precision": prec,
            "backward": backward, "estimate": float(it.est[-1].item()), "data": "synthetic",
            "l2": "flushed before every timed step (512 MiB write, untimed)",
            "kernels": {k: {"launches": c // args.steps, "ms_per_step": t / args.steps}
                        for k, (c, t) in sorted(kern.items())}}


def main():
    args = parse()
    if args.workload != "c2" and args.impl == "ours":
        print(json.dumps(run_workload(args)))
        return
    dist, rank, world = dist_setup(args)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, dist, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
