"""Benchmark of the reduced QMC matrix-vector product on one GB300 (or N replicas).

A step is one pass of the whole hot path over the reduced digital-net workload (b=2, m=20 ->
N=1048576 points, s=tau=1024, w_j=min(floor(log2(j+1)),12), C_j=[[B_j,0],[0,0]] with B_j a
random nonsingular GF(2) block, A ~ N(0,1/s) in FP32, 16 random 32-bit digital shifts,
f(y)=exp(-|y|^2/(2 tau))): point generation and shifts, the coarse block products on the
distinct rows, the periodic broadcast-accumulate fused with f and the mean, and the folded
adjoint dQ/dA, for all 16 shifts in one call each.
Metric: x_k^T A outputs per second, N*tau*R / step time.  The headline tier is the split
tier (bf16x6 tensor-core block products, FP32 elsewhere); the FP32 and plain-bf16 tiers are
timed beside it, with the dense X*A on the same GPU (FP32, BF16 and the three-product split
BF16 GEMMs of torch) and the oracle on the host cores.  The Gaussian-expectation lattice
(m=16, s=tau=512) and the adjoint lattice (m=20, s=tau=1024, R=8, log-sum-exp) are timed as
extra keys.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision split|fp32|bf16] [--workload net20|gauss16|adjoint20|basket]
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
TIERS = ("split", "fp32", "bf16")
GOLDEN = os.path.join(ROOT, "tests", "golden", "full_size_oracle.json")
# dram__bytes_read.sum + dram__bytes_write.sum per launch, scaled to the contract workload from
# the ncu captures summarised under profiles/ (workload name, kernel name); a kernel missing
# here has changed since its counters were taken and reports traffic null
TRAFFIC_BYTES = {
    # profiles/net20_top_kernels.md: the 2-shift capture of the 16-shift contract workload, scaled by
    # 16/2 (each shift's data are separate, so the DRAM bytes grow with the shifts)
    ("net20", "k_fine_bwd_s4"): (590.064384e6 + 500.344064e6) * 8,
    ("net20", "k_fold_grad_tc"): (576.025088e6 + 60.776704e6) * 8,
    ("net20", "k_grad_tc"): (166.576384e6 + 3.463936e6) * 8,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=list(TIERS), default="split")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense X*A comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    ap.add_argument("--no-tiers", action="store_true", help="time only the requested precision tier")
    ap.add_argument("--no-mat", action="store_true", help="skip the materialised product")
    ap.add_argument("--shifts", type=int, default=0,
                    help="keep only the first R shifts of the workload (smaller profiler captures; not the "
                         "contract line)")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="net20",
                    help="net20: the contract line (default); the others time one workload alone")
    return ap.parse_args()


# ----------------------------------------------------------------------------- workloads

def _basket():
    from paper_2305_11645_gb300 import inputs as I
    m, s = 25, 10
    sig, rho, S0, K = 0.4, 0.2, 100.0, 110.0
    Sig = np.diag([sig] * s) + np.diag([rho] * (s - 1), 1) + np.diag([rho] * (s - 1), -1)
    A = np.linalg.cholesky(Sig).T.astype(np.float32)
    w = np.array([min(int(math.floor(math.log2(j))), m) for j in range(1, s + 1)], dtype=np.uint32)
    y = I.mc_samples(I.rng(6, I.P_MISC), m, w, 1, force_odd=True)
    return I.Problem(I.REDUCED_MC, m, w, A, y=y, transform=I.T_INV_NORMAL, f_kind=I.F_CALL_MEAN_EXP,
                     f_params=(1.0, K / S0 * math.exp(sig / 2), 0, 0), name="basket")


def _make(name):
    from paper_2305_11645_gb300 import inputs as I
    if name == "pde8":
        return [I.c4(i) for i in range(len(I.C4_INSTANCES))]
    if name == "pde_asm":
        return I.pde_assembly(m=18, s=256, M=32, R=1)
    return {"net20": I.c3, "gauss16": lambda: I.c2(dtype=np.float32), "adjoint20": I.c5, "basket": _basket}[name]()


# name -> (step includes the adjoint, golden key, description)
WORKLOADS = {
    "net20": (True, "c3", "reduced periodic digital net b=2 m=20 (N=1048576), s=tau=1024, "
                          "w_j=min(floor(log2(j+1)),12), C_j=[[B_j,0],[0,0]] (B_j random nonsingular over GF(2)), "
                          "A~N(0,1/s) FP32, R=16 random 32-bit digital shifts, f=exp(-|y|^2/(2 tau)); "
                          "estimate + adjoint dQ/dA"),
    "gauss16": (True, None, "Gaussian expectation: reduced rank-1 lattice b=2 m=16 (N=65536), s=tau=512, "
                            "w_j=min(floor(log2(j+1)),10), 1 odd 32-bit shift, inverse-normal transform, A=L^T "
                            "(exp covariance), f=max(mean exp(0.2y)-1,0); estimate + adjoint"),
    "adjoint20": (True, "c5", "reduced rank-1 lattice b=2 m=20 (N=1048576), s=tau=1024, "
                              "w_j=min(floor(log2(j+1)),12), A~N(0,1/s) FP32, R=8 shifts, f=log sum exp(y); "
                              "estimate + adjoint"),
    "pde8": (False, "c4", "8 uneven PDE-like reduced lattice instances (m, s, tau) = (14,256,1024), (14,2048,4096), "
                          "(16,1024,2048), (16,256,4096), (16,2048,1024), (18,1024,1024), (18,256,2048), "
                          "(18,2048,4096), w_j=min(floor(log2(j+1)),12), centred points, 4 shifts each, "
                          "A_ji=(j+1)^-2 sin((j+1) pi t_i), f=mean (1+0.5y)^-2; schedules autotuned per instance, "
                          "all instances in one call replayed as one CUDA graph; estimate"),
    "pde_asm": (False, None, "PDE matrix assembly D_k = sum_j x_{j,k} C_j (Sec. 1) as the materialised reduced "
                             "product: reduced lattice b=2 m=18 (N=262144), s=256 stiffness terms of M=32 interior "
                             "nodes (tau=M^2=1024), w_j=min(floor(log2(j+1)),12), one shift; D written as N x M x M "
                             "FP32"),
    "basket": (False, None, "basket option by reduced Monte Carlo: m=25 (N=33554432), s=tau=10, "
                            "w_j=floor(log2 j) (1-based), tridiagonal Sigma (0.4, 0.2), K=110, one replica; estimate"),
}


def golden(key):
    """The oracle's stored full-size values (written by tests/golden/make_full_size.py), or None."""
    if key is None or not os.path.exists(GOLDEN):
        return None
    with open(GOLDEN) as fh:
        return json.load(fh).get(key)


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


# ----------------------------------------------------------------------------- work models

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


# FP32-pipe operations (an FMA counts once) and MUFU operations of h(y) per output, with the
# row accumulation: linear u += v; cos: MUFU cos, add; call: MUFU ex2, add; Gaussian norm:
# u = fma(v, v, u); inverse square: fma(c, v, 1), MUFU rcp, fma(r, r, u); log-sum-exp: the
# difference to the running maximum, MUFU ex2, the select/fma and the maximum
H_OPS = {1: (1, 0), 2: (1, 1), 3: (1, 1), 4: (1, 0), 5: (2, 1), 6: (3, 1)}
# MUFU (ex2, sin, cos, rcp) lanes per SM per clock: ncu's peak for the XU pipe is one warp
# instruction per 4 cycles per SM sub-partition (measured: an ex2 loop reaches 27.6 per clock)
MUFU_LANES = 32


def fine_work(p, name):
    """Algorithmic work of the fine-band (S4) kernels per step, counted per output of all shifts:
    the tree's multiply-adds sum_{I<4} tau_I 2^-I (4 for a full band) and h(y) with the row
    accumulation (forward); the recomputed tree, G = coef h'(y) (h' and a multiply), the fold
    (one add per output amortised) and the gradient multiply-adds (adjoint: twice the tree).
    Returns (FP32 pipe operations, MUFU operations)."""
    jf, tau_I, _ = band_of(p)
    outs = p.N * p.tau * p.R_eff
    fma = sum(tau_I[I] / 2.0 ** I for I in range(jf))
    fp_h, mufu_h = H_OPS[p.f_kind]
    per = (fma + fp_h) if "fwd" in name else (2 * fma + fp_h + 2)
    return outs * per, outs * mufu_h


def coarse_mma_flops(p, pieces, levels=None):
    """MMA flops of the coarse block products of one step (forward X_I A_I or adjoint X_I^T F_I, the
    same contraction sizes): 2 n_I tau tau_I per coarse level I (n_I = 2^(m-I) distinct rows), for
    every shift, times the piece products (6 in the split tier, 1 in the bf16 tier); every coarse
    level, or the given ones."""
    jf, tau_I, chain = band_of(p)
    np_ = 6 if pieces == 3 else 1
    lv = chain if levels is None else levels
    return sum(2.0 * 2 ** (p.m - I) * p.tau * tau_I[I] for I in lv) * p.R_eff * np_


def coarse_kernel_levels(p, name):
    """The coarse levels whose block products a tensor-core kernel computes, as the library's
    planner assigns them: k_level_tc every coarse level (forward); k_fold_grad_tc the L <= 3 lowest
    ones (adjoint, one entry of at most 128 columns each, 128 columns in all, at least 32 distinct
    rows left at level JF+L, which lies within six folds of JF and below m); k_grad_tc the other
    levels with at least 32 distinct rows whose folded gradient is materialised; k_coarse_grad_tc the
    rest."""
    jf, tau_I, chain = band_of(p)
    if name == "k_level_tc":
        return chain
    below = [I for I in chain if I < p.m and I - jf <= 6]
    i_mat = max(below) if below else jf
    fused = []
    for L in (3, 2, 1):
        if jf + L > i_mat or p.m - (jf + L) < 5:
            continue
        lv = [I for I in range(jf, jf + L)]
        cols = sum((tau_I[I] + 15) // 16 * 16 for I in lv)
        if any(tau_I[I] > 128 for I in lv) or cols > 128 or cols == 0:
            continue
        fused = [I for I in lv if tau_I[I] > 0]
        break
    rest = [I for I in chain if I not in fused]
    tma = [I for I in rest if p.m - I >= 5 and I <= i_mat]
    if name == "k_fold_grad_tc":
        return fused
    if name == "k_grad_tc":
        return tma
    return [I for I in rest if I not in tma]


def tensor_roofline(flops, seconds, peak_tflops):
    return {"bound": "tensor", "achieved": flops / seconds / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": flops / seconds / 1e12 / peak_tflops}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        return mp, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


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


def roofline_of(p, prec, name, ms_per_step, launches_per_step, clk, mp, peak_src, workload=None):
    """Roofline of one kernel from its device time per step (the sum over its launches; its
    algorithmic work per step is the sum over the same launches)."""
    sec = ms_per_step / 1e3
    if name.endswith("_tc"):
        fl = coarse_mma_flops(p, 3 if prec == "split" else 1, coarse_kernel_levels(p, name))
        r = tensor_roofline(fl, sec, mp["bf16_tflops_sustained"])
        r["peak_source"] = (f"{peak_src} dense bf16 sustained peak (MEASURED_PEAKS.json bf16_tflops_sustained: "
                            f"the kernel runs inside a long step)")
        r["work"] = {"mma_flops_per_step": fl}
    else:
        w32, wmu = fine_work(p, name)
        r = alu_roofline(w32, wmu, sec, clk)
        r["peak_source"] = (f"derived: {SM_COUNT} SMs x pipe lanes (FP32 128, MUFU {MUFU_LANES}) x median SM "
                            f"clock {clk:.0f} MHz sampled during the timed region")
        r["work"] = {"fp32_ops_per_step": w32, "mufu_ops_per_step": wmu}
    tb = TRAFFIC_BYTES.get((workload, name))
    r.update({"kernel": name, "ms_per_step": ms_per_step, "launches_per_step": launches_per_step,
              "traffic": None if tb is None else tb / max(launches_per_step, 1.0)})
    return r


# ----------------------------------------------------------------------------- timing helpers

class Timer:
    """CUDA-event timing of a step on the launching stream, with L2 flushed before every step."""

    def __init__(self, dev, dist):
        self.dev, self.dist = dev, dist
        self.stream = torch.cuda.current_stream(dev)
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def run(self, fn, steps, trace=False, prequeue=False):
        from paper_2305_11645_gb300 import _lib as L
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(self.dist)
        torch.cuda.synchronize()
        if trace:
            L.trace_enable(True)
        for a, b in evs:
            self.flush.zero_()
            if prequeue:
                torch.cuda._sleep(3_000_000)    # the host queues the whole step before the GPU reaches it
            a.record(self.stream)
            fn()
            b.record(self.stream)
        torch.cuda.synchronize()
        barrier(self.dist)
        kern = None
        if trace:
            L.trace_enable(False)
            kern = L.trace_collect()
        return [a.elapsed_time(b) for a, b in evs], kern


def measure(p, prec, backward, timer, steps, warmup):
    """The graph-replayed step of one workload: mean ms, and the per-kernel device times of the same
    steps launched eagerly with the library's kernel trace."""
    from paper_2305_11645_gb300 import api
    dev = timer.dev
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(np.ascontiguousarray(p.A)).to(dev)
    f = api.Integrand(p.f_kind, p.f_params)
    integ = api.Integrator(rule, A, f, backward=backward, graph=True, precision=prec)
    eager = api.Integrator(rule, A, f, backward=backward, graph=False, precision=prec)
    for _ in range(warmup):
        integ.run()
        eager.run()
    torch.cuda.synchronize()
    times, _ = timer.run(integ.run, steps)
    _, kern = timer.run(eager.run, steps, trace=True, prequeue=True)
    del eager
    kernels = {k: {"launches_per_step": c / steps, "ms_per_step": t / steps} for k, (c, t) in sorted(kern.items())}
    return integ, statistics.mean(times), kernels, sum(c for c, _ in kern.values()) / steps


def measure_batch(ps, prec, timer, steps, warmup, tune=True):
    """Several problems in one call (the library runs them on parallel internal streams), replayed as
    one CUDA graph; each instance's fine schedules autotuned first.  Returns the integrator, mean ms
    per step, the per-kernel device times (eager, traced) and the timed candidates."""
    from paper_2305_11645_gb300 import api
    dev = timer.dev
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(np.ascontiguousarray(p.A)).to(dev) for p in ps]
    fs = [api.Integrand(p.f_kind, p.f_params) for p in ps]
    timed = sum(api.autotune(r, a, f, precision=prec) for r, a, f in zip(rules, As, fs)) if tune else 0
    integ = api.Integrator(rules, As, fs, backward=False, graph=True, precision=prec)
    eager = api.Integrator(rules, As, fs, backward=False, graph=False, precision=prec)
    for _ in range(warmup):
        integ.run()
        eager.run()
    torch.cuda.synchronize()
    times, _ = timer.run(integ.run, steps)
    _, kern = timer.run(eager.run, steps, trace=True)
    del eager
    kernels = {k: {"launches_per_step": c / steps, "ms_per_step": t / steps} for k, (c, t) in sorted(kern.items())}
    return integ, statistics.mean(times), kernels, timed


def batch_accuracy(ps, est, tier):
    g = golden("c4")
    if g is None:
        return {}
    e = est.cpu().numpy()
    off, worst = 0, 0.0
    for i, p in enumerate(ps):
        worst = max(worst, abs(float(e[off + p.R_eff]) - g[i]["mean"]) / abs(g[i]["mean"]))
        off += p.R_eff + 1
    return {"max_instance_estimate_rel_err": worst, "tolerance": {"split": 1e-6, "fp32": 2e-5, "bf16": 2e-3}[tier]}


def accuracy(key, p, est, grad, tier):
    """Errors against the oracle's stored full-size values: the mean estimate (relative) and, where
    stored, the gradient (max-norm relative)."""
    g = golden(key)
    if g is None:
        return {"estimate": float(est[-1]), "oracle": None}
    e = est.cpu().numpy()
    out = {"estimate": float(e[-1]), "oracle_estimate": g["mean"],
           "estimate_rel_err": abs(float(e[-1]) - g["mean"]) / abs(g["mean"]),
           "per_shift_max_rel_err": float(np.max(np.abs(e[:-1] - np.array(g["Q"])) / np.abs(np.array(g["Q"]))))}
    if grad is not None and g.get("grad_file"):
        G = np.load(os.path.join(os.path.dirname(GOLDEN), g["grad_file"])).astype(np.float64)
        out["grad_rel_err"] = float(np.max(np.abs(grad.double().cpu().numpy() - G)) / np.max(np.abs(G)))
    out["tolerance"] = {"split": 1e-6, "fp32": 2e-5, "bf16": 2e-3}[tier]
    return out


# ----------------------------------------------------------------------------- our arm

def run_batch(args, dist, world, timer):
    """The uneven batch (pde8) alone: one line with its step time, kernels and accuracy."""
    ps = _make("pde8")
    prec = args.precision
    clocks = ClockSampler(timer.dev.index)
    clocks.start()
    time.sleep(0.3)
    integ, ms, kernels, ntimed = measure_batch(ps, prec, timer, args.steps, args.warmup)
    clock_info = clocks.stop()
    est = integ.run()[0]
    torch.cuda.synchronize()
    ms_max = max_over_ranks(dist, ms)
    outputs = sum(q.N * q.tau * q.R_eff for q in ps)
    return {"metric": METRIC, "value": world * outputs / (ms_max / 1e3), "unit": "outputs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"split": "bf16x6+f32", "fp32": "f32", "bf16": "bf16+f32"}[prec],
            "data": "synthetic", "config": {"workload": WORKLOADS["pde8"][2], "name": "pde8",
                                            "outputs_per_step": outputs, "precision": prec,
                                            "l2": "flushed before every timed step (512 MiB write, untimed)"},
            "autotune_candidates_timed": ntimed, "kernels": kernels, "clocks": clock_info,
            "gpu_launches": int(round(sum(k["launches_per_step"] for k in kernels.values()) * args.steps)),
            "accuracy": batch_accuracy(ps, est, prec)}


def run_assembly(args, dist, world, timer):
    """Sec. 1's PDE assembly alone: D = X A written to HBM (api.assemble), its band kernel's share of
    the measured copy bandwidth, and the oracle's matrices on sampled points."""
    from paper_2305_11645_gb300 import api
    from paper_2305_11645_gb300 import inputs as I
    from paper_2305_11645_gb300 import _lib as L
    p = _make("pde_asm")
    M = 32
    prec = args.precision
    rule = api.Rule.from_problem(p)
    C = torch.from_numpy(I.stiffness_terms(p.s, M).astype(np.float32)).to(timer.dev)
    ws = torch.empty(max(api.workspace_size(L.QMC_OP_REDUCED_MATMUL, [rule], [M * M], None,
                                            api._precision(C.reshape(p.s, -1), prec)), 256),
                     dtype=torch.uint8, device=timer.dev)
    for _ in range(args.warmup):
        D = api.assemble(rule, C, ws=ws, precision=prec)
    torch.cuda.synchronize()
    clocks = ClockSampler(timer.dev.index)
    clocks.start()
    time.sleep(0.3)
    times, _ = timer.run(lambda: api.assemble(rule, C, ws=ws, precision=prec), args.steps)
    clock_info = clocks.stop()
    _, kern = timer.run(lambda: api.assemble(rule, C, ws=ws, precision=prec), args.steps, trace=True)
    ms = max_over_ranks(dist, statistics.mean(times))
    outputs = p.N * M * M * p.R_eff
    D = api.assemble(rule, C, ws=ws, precision=prec)
    torch.cuda.synchronize()
    ks = np.array([0, 1, 12345, p.N - 1])
    want = O_assemble(p, I.stiffness_terms(p.s, M).astype(np.float32).astype(np.float64), ks)
    got = D[0][torch.from_numpy(ks).to(timer.dev)].double().cpu().numpy()
    mp, peak_src = peaks()
    band = "k_fine_mat_s4"
    roof = None
    if band in kern:
        cnt, tot = kern[band]
        sec = tot / cnt / 1e3
        roof = {"bound": "hbm", "kernel": band, "achieved": outputs * 4 / sec / 1e9, "peak": mp["hbm_gbs"],
                "unit": "GB/s", "frac": outputs * 4 / sec / 1e9 / mp["hbm_gbs"], "bytes_per_launch": outputs * 4,
                "traffic": None, "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    return {"metric": METRIC, "value": world * outputs / (ms / 1e3), "unit": "outputs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"split": "bf16x6+f32", "fp32": "f32", "bf16": "bf16+f32"}[prec],
            "data": "synthetic", "config": {"workload": WORKLOADS["pde_asm"][2], "name": "pde_asm",
                                            "outputs_per_step": outputs, "precision": prec},
            "roofline": roof, "clocks": clock_info,
            "kernels": {k: {"launches": c / args.steps, "ms_per_step": t / args.steps} for k, (c, t) in sorted(kern.items())},
            "accuracy": {"sampled_rows_max_rel_err": float(np.max(np.abs(got - want)) / np.max(np.abs(want)))}}


def O_assemble(p, C, ks):
    from oracle import qmc_oracle as O
    return O.assemble(p, C, 0, ks)


def run_ours(args, dist, rank, world):
    from paper_2305_11645_gb300 import _lib as L
    from paper_2305_11645_gb300 import api
    from paper_2305_11645_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(dist)
    dev = torch.device("cuda", torch.cuda.current_device())
    timer = Timer(dev, dist)
    name = args.workload
    if name == "pde8":
        return run_batch(args, dist, world, timer)
    if name == "pde_asm":
        return run_assembly(args, dist, world, timer)
    backward, gkey, desc = WORKLOADS[name]
    p = _make(name)
    if args.shifts and p.shifts is not None:
        import dataclasses
        p = dataclasses.replace(p, shifts=p.shifts[:args.shifts])
        gkey = None
        desc += f" (first {p.R_eff} shifts only)"
    prec = args.precision
    outputs = p.N * p.tau * p.R_eff

    # the contract step: one CUDA graph of the forward and backward launches (api.Integrator)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    integ, ms, kernels, launches = measure(p, prec, backward, timer, args.steps, args.warmup)
    clock_info = clocks.stop()
    ms_max = max_over_ranks(dist, ms)
    value = world * outputs / (ms_max / 1e3)
    est, grad = integ.run()
    torch.cuda.synchronize()

    mp, peak_src = peaks()
    clk = clock_info["sm_mhz"] or mp.get("sm_max_mhz", 2070.0)
    top = max(kernels.items(), key=lambda kv: kv[1]["ms_per_step"])
    roof = roofline_of(p, prec, top[0], top[1]["ms_per_step"], top[1]["launches_per_step"], clk, mp, peak_src,
                       None if args.shifts else name)
    kernel_total = sum(k["ms_per_step"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = k["ms_per_step"] / kernel_total
    # every kernel's roofline fraction, and the whole step's: the ALU, tensor and MUFU work of the
    # step at full rate against the graph-replayed step time
    per_kernel = {}
    for k, v in kernels.items():
        if k.startswith("k_fine_") and "mat" not in k:
            per_kernel[k] = roofline_of(p, prec, k, v["ms_per_step"], v["launches_per_step"], clk, mp, peak_src)["frac"]
        elif k.endswith("_tc"):
            per_kernel[k] = roofline_of(p, prec, k, v["ms_per_step"], v["launches_per_step"], clk, mp, peak_src)["frac"]
    roof["per_kernel_frac"] = per_kernel
    # the whole step against its compute roofline: every fine-band FP32 operation at the FP32 pipe's
    # peak plus every block-product flop at the sustained tensor peak (the HBM traffic of the root
    # values and the folds is reported beside it, not added)
    pieces = 3 if prec == "split" else 1
    f32 = fine_work(p, "fwd")[0] + (fine_work(p, "bwd")[0] if backward else 0.0)
    mma = coarse_mma_flops(p, pieces) * (2 if backward else 1) if prec in ("split", "bf16") else 0.0
    t_f32 = f32 / (SM_COUNT * 128 * clk * 1e6)
    t_mma = mma / (mp["bf16_tflops_sustained"] * 1e12)
    jf, tau_I, chain = band_of(p)
    root_bytes = p.R_eff * 2 ** (p.m - jf) * p.tau * 4.0
    roof["step"] = {"fp32_ms": t_f32 * 1e3, "tensor_ms": t_mma * 1e3, "frac": (t_f32 + t_mma) / (ms / 1e3),
                    "root_value_hbm_ms": (2 if not backward else 6) * root_bytes / (mp["hbm_gbs"] * 1e9) * 1e3,
                    "note": "FP32 ops of the fine band at 152x128 lanes x clock plus block-product MMA flops at the "
                            "measured sustained bf16 peak, over the graph-replayed step time; root_value_hbm_ms is "
                            "the root values written and read (and, with the adjoint, the root gradients and their "
                            "folds) at the measured copy bandwidth"}

    # end to end through the public API with host buffers: H2D of A, D2H of the estimates and dQ/dA
    A_host = torch.from_numpy(np.ascontiguousarray(p.A)).pin_memory()
    est_host = torch.empty(p.R_eff + 1, dtype=torch.float64).pin_memory()
    grad_host = torch.empty(p.A.shape, dtype=torch.float32).pin_memory()

    def e2e_step():
        integ.A.copy_(A_host, non_blocking=True)
        e, g = integ.run()
        est_host.copy_(e, non_blocking=True)
        if backward:
            grad_host.copy_(g, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    for _ in range(2):
        e2e_step()
    etimes, _ = timer.run(e2e_step, args.steps)
    e_ms = max_over_ranks(dist, statistics.mean(etimes))
    e2e = {"value": world * outputs / (e_ms / 1e3), "unit": "outputs/s", "ms_per_step": e_ms,
           "h2d_bytes_per_step": int(A_host.numel() * 4),
           "d2h_bytes_per_step": int(est_host.numel() * 8 + (grad_host.numel() * 4 if backward else 0))}

    result = {"metric": METRIC, "value": value, "unit": "outputs/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": {"split": "bf16x6+f32", "fp32": "f32", "bf16": "bf16+f32"}[prec],
              "data": "synthetic",
              "config": {"workload": desc, "name": name, "N": p.N, "s": p.s, "tau": p.tau, "R": p.R_eff,
                         "outputs_per_step": outputs, "precision": prec,
                         "step": ("qmc_integrate + qmc_integrate_backward (reusing the forward's workspace)"
                                  if backward else "qmc_integrate") + ", replayed as one CUDA graph (api.Integrator)",
                         "l2": "flushed before every timed step (512 MiB write, untimed)",
                         "parallelism": "replicas" if world > 1 else "single"},
              "roofline": roof, "e2e": e2e, "gpu_launches": int(round(launches * args.steps)), "clocks": clock_info,
              "kernels": kernels, "peaks": peak_src}
    del integ
    torch.cuda.empty_cache()

    if rank == 0:
        result["accuracy"] = accuracy(gkey, p, est, grad if backward else None, prec)
        tiers = {prec: {"ms_per_step": ms, "value": outputs / (ms / 1e3), **result["accuracy"]}}
        for t in TIERS:
            if t == prec or args.no_tiers:
                continue
            it, t_ms, t_k, _ = measure(p, t, backward, timer, max(3, args.steps // 2), 2)
            e_t, g_t = it.run()
            torch.cuda.synchronize()
            tiers[t] = {"ms_per_step": t_ms, "value": outputs / (t_ms / 1e3),
                        "kernels": {k: v["ms_per_step"] for k, v in t_k.items()},
                        **accuracy(gkey, p, e_t, g_t if backward else None, t)}
            del it
            torch.cuda.empty_cache()
        result["tiers"] = tiers
        if not args.no_mat:
            result["materialized"] = materialized_product(p, prec, timer, args)
        if not args.no_dense:
            result["dense_xa"] = dense_baseline(p, gkey, backward, timer, args)
        if not args.no_extra:
            extra = {}
            ps8 = _make("pde8")
            it, b_ms, b_k, b_n = measure_batch(ps8, prec, timer, max(5, args.steps // 2), 3)
            e_b = it.run()[0]
            torch.cuda.synchronize()
            outs8 = sum(q.N * q.tau * q.R_eff for q in ps8)
            extra["pde8"] = {"workload": WORKLOADS["pde8"][2], "ms_per_step": b_ms, "value": outs8 / (b_ms / 1e3),
                             "unit": "outputs/s", "autotune_candidates_timed": b_n,
                             "kernels": {k: v["ms_per_step"] for k, v in b_k.items()}, **batch_accuracy(ps8, e_b, prec)}
            del it
            torch.cuda.empty_cache()
            for nm in ("gauss16", "adjoint20"):
                if nm == name:
                    continue
                q = _make(nm)
                bw, gk, d = WORKLOADS[nm]
                it, q_ms, q_k, _ = measure(q, prec, bw, timer, max(5, args.steps // 2), 3)
                e_q, g_q = it.run()
                torch.cuda.synchronize()
                extra[nm] = {"workload": d, "ms_per_step": q_ms, "value": q.N * q.tau * q.R_eff / (q_ms / 1e3),
                             "unit": "outputs/s", "kernels": {k: v["ms_per_step"] for k, v in q_k.items()},
                             **accuracy(gk, q, e_q, g_q if bw else None, prec)}
                del it
                torch.cuda.empty_cache()
            result["extra_workloads"] = extra
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(p, budget_s=12.0)
    return result


def materialized_product(p, prec, timer, args):
    """The materialised product P = X A of the workload's shape (qmc_reduced_matmul) for its first two
    shifts (2 x N x tau FP32 outputs): the band kernel is bound by its output writes, 4 bytes per
    output (the root values and the point table it reads are under 5 % of that)."""
    from paper_2305_11645_gb300 import _lib as L
    from paper_2305_11645_gb300 import api
    from paper_2305_11645_gb300 import inputs as I
    import dataclasses
    q = dataclasses.replace(p, shifts=None if p.shifts is None else p.shifts[:2])
    rule = api.Rule.from_problem(q)
    A = torch.from_numpy(np.ascontiguousarray(q.A)).to(timer.dev)
    mws = torch.empty(max(api.workspace_size(L.QMC_OP_REDUCED_MATMUL, [rule], [q.tau], None,
                                             api._precision(A, prec)), 256), dtype=torch.uint8, device=timer.dev)
    P = torch.empty((q.R_eff, q.N, q.tau), dtype=torch.float32, device=timer.dev)

    def call():
        api.reduced_matmul(rule, A, ws=mws, precision=prec, out=P)

    for _ in range(3):
        call()
    steps = max(3, args.steps // 2)
    ms = statistics.mean(timer.run(call, steps)[0])
    _, kern = timer.run(call, steps, trace=True, prequeue=True)
    outputs = q.N * q.tau * q.R_eff
    mp, peak_src = peaks()
    res = {"op": f"qmc_reduced_matmul (P = X A, {q.R_eff} x N x tau float32, the workload's first shifts)",
           "ms_per_call": ms, "value": outputs / (ms / 1e3), "unit": "outputs/s",
           "kernels": {k: {"launches": c / steps, "ms_per_call": t / steps} for k, (c, t) in sorted(kern.items())}}
    band = "k_fine_mat_s4" if "k_fine_mat_s4" in kern else "k_fine_fwd_materialize"
    if band in kern:
        cnt, tot = kern[band]
        sec = tot / cnt / 1e3
        res["roofline"] = {"bound": "hbm", "kernel": band, "achieved": outputs * 4 / sec / 1e9, "peak": mp["hbm_gbs"],
                           "unit": "GB/s", "frac": outputs * 4 / sec / 1e9 / mp["hbm_gbs"],
                           "bytes_per_launch": outputs * 4, "launch_ms": sec * 1e3, "traffic": None,
                           "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    res["whole_call_hbm_frac"] = outputs * 4 / (ms / 1e3) / 1e9 / mp["hbm_gbs"]
    del P, mws
    torch.cuda.empty_cache()
    return res


def torch_integrand(kind, params, Y, tau):
    """f per row and df/dy of the QMC_F_* integrands, in torch (the dense baseline's epilogue)."""
    c, K = params[0], params[1]
    Y = Y.float()
    if kind == 4:                                             # Gaussian norm
        fv = torch.exp(-(Y * Y).sum(dim=1) / (2.0 * tau))
        return fv, -fv[:, None] * Y / tau
    if kind == 3:                                             # call on the mean exponential
        E = torch.exp(c * Y)
        m_ = E.mean(dim=1)
        return torch.clamp(m_ - K, min=0.0), (c * E / tau) * (m_ > K).float()[:, None]
    if kind == 6:                                             # log-sum-exp
        return torch.logsumexp(Y, dim=1), torch.softmax(Y, dim=1)
    if kind == 5:
        r = 1.0 / (1.0 + c * Y)
        return (r * r).mean(dim=1), -2.0 * c * r ** 3 / tau
    if kind == 2:
        return torch.cos(Y).mean(dim=1), -torch.sin(Y) / tau
    return Y.mean(dim=1), torch.full_like(Y, 1.0 / tau)


def dense_baseline(p, gkey, backward, timer, args):
    """Dense X*A on the same GPU for the first shift: X materialised once by gen_points (untimed),
    then per step Y = X A (torch GEMM), f, the mean and dQ/dA = X^T G, in FP32 (TF32 off), BF16, and
    the three-product split BF16 of the 1e-6 tier (hi/lo bf16 pieces of X, A and G, products
    hi*hi + hi*lo + lo*hi accumulated in FP32 by torch.mm(..., out_dtype=float32)).  Outputs per
    second count the N x tau outputs of one shift."""
    from paper_2305_11645_gb300 import api
    dev = timer.dev
    rule = api.Rule.from_problem(p)
    x32 = api.gen_points(rule, "full", 0, device=dev).to(torch.int64) & 0xFFFFFFFF
    X = x32.double().mul_(2.0 ** -32)
    del x32
    if p.transform == 2:
        X = torch.special.ndtri(X)
    elif p.transform == 1:
        X = X - 0.5
    X = X.float()
    A = torch.from_numpy(np.ascontiguousarray(p.A)).to(dev).float()
    g = golden(gkey)
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False

    def split(T):
        hi = T.to(torch.bfloat16)
        return hi, (T - hi.float()).to(torch.bfloat16)

    def mm3(a, b):
        ah, al = a
        bh, bl = b
        return (torch.mm(ah, bh, out_dtype=torch.float32) + torch.mm(ah, bl, out_dtype=torch.float32)
                + torch.mm(al, bh, out_dtype=torch.float32))

    for name in ("fp32", "bf16", "split3_bf16"):
        if name == "split3_bf16":
            try:
                torch.mm(X[:8, :8].to(torch.bfloat16), A[:8, :8].to(torch.bfloat16), out_dtype=torch.float32)
            except (TypeError, RuntimeError) as e:
                out[name] = {"unavailable": f"torch.mm(..., out_dtype=float32) on bf16: {type(e).__name__}"}
                continue
            Xs, As_ = split(X), split(A)
            XsT = (Xs[0].t().contiguous(), Xs[1].t().contiguous())

            def step():
                Y = mm3(Xs, As_)
                fv, G = torch_integrand(p.f_kind, p.f_params, Y, p.tau)
                est = fv.double().mean()
                grad = mm3(XsT, split(G / p.N)) if backward else None
                return est, grad
        else:
            dt = torch.float32 if name == "fp32" else torch.bfloat16
            Xd, Ad = X.to(dt), A.to(dt)
            XdT = Xd.t().contiguous()

            def step():
                Y = Xd @ Ad
                fv, G = torch_integrand(p.f_kind, p.f_params, Y, p.tau)
                est = fv.double().mean()
                grad = (XdT @ (G / p.N).to(dt)) if backward else None
                return est, grad

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, args.steps // 4)):
            timer.flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(timer.stream)
            est, grad = step()
            b.record(timer.stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.mean(ts)
        res = {"value": p.N * p.tau / (ms / 1e3), "unit": "outputs/s", "ms_per_shift": ms,
               "estimate_shift0": est.item()}
        if g is not None:
            res["estimate_rel_err"] = abs(est.item() - g["Q"][0]) / abs(g["Q"][0])
        out[name] = res
        torch.cuda.empty_cache()
    torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def oracle_sample(p, ks):
    """The oracle on the rows ks of every shift: points from the definitions, X A, f and X^T grad f."""
    from oracle import qmc_oracle as O
    for r, X in O.shifted_rows(p, ks):
        Y = O.product(X, p.A)
        if p.f_kind == 0:                          # the product alone (the assembly workload)
            continue
        O.integrand(p.f_kind, p.f_params, Y).sum()
        X.T @ O.integrand_grad(p.f_kind, p.f_params, Y)


def cpu_baseline(p, budget_s: float = 12.0, rows: int = 512):
    """The oracle as it stands (numpy FP64) on a bounded sample of the workload: blocks of rows of
    every shift, until the time budget is spent."""
    done = 0
    t0 = time.perf_counter()
    while True:
        ks = (np.arange(rows, dtype=np.int64) + done) % p.N
        oracle_sample(p, ks)
        done += rows
        el = time.perf_counter() - t0
        if el >= budget_s or done >= p.N:
            break
    cores = len(os.sched_getaffinity(0))
    return {"value": done * p.tau * p.R_eff / el, "unit": "outputs/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of {p.N} rows of the workload for all {p.R_eff} shifts: points from the definitions, "
                      f"X A, f and X^T grad f in numpy FP64 (BLAS may use up to {cores} threads, the rest one "
                      f"thread), {el:.1f} s"}


# ----------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return None
    name = getattr(args, "workload", "net20")
    ps = _make(name)
    ps = ps if isinstance(ps, list) else [ps]
    backward, _, desc = WORKLOADS[name]
    rows = 256 // len(ps)

    def step(i):
        for p in ps:
            oracle_sample(p, (np.arange(rows, dtype=np.int64) + i * rows) % p.N)

    for i in range(args.warmup):
        step(i)
    ts = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + i)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(ts)
    value = sum(rows * p.tau * p.R_eff for p in ps) / (ms / 1e3)
    cores = len(os.sched_getaffinity(0))
    p = ps[0]
    sample = (f"{rows} rows of {'each instance of ' if len(ps) > 1 else ''}the workload per step for all shifts, "
              f"numpy FP64 oracle: points from the definitions, X A, f and X^T grad f")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "outputs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc + "; bounded row sample per step", "name": name, "N": p.N, "s": p.s,
                       "tau": p.tau, "R": p.R_eff, "rows_per_step": rows},
            "cpu_baseline": {"value": value, "unit": "outputs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "outputs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
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
