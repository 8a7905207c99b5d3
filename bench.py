"""Benchmark: FP64 block-oriented one-sided Jacobi SVD on one GB300.

A step is one complete SVD (all block sweeps to convergence, plus U, S, V)
of one synthetic matrix already resident in HBM.  The default workload is
the 8192 x 8192 graded Gaussian (N(0,1) entries, column j scaled by 10^u_j,
u_j ~ U(-4, 0)), block width b = 32, reverse row-cyclic-closest p-strategy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference      # the CPU oracle on a bounded sample

Prints one JSON line (rank 0).  value = seconds per matrix for the whole job
(time of the slowest rank / matrices processed by all ranks); ranks solve
independent matrices (replicas, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 Jacobi SVD s/matrix at 8192²; TFLOP/s vs DMMA peak; mixed vs plain at 1e-12"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
NOMINAL_BF16_TF = 2250.0
NOMINAL_FP64_TF = 1.25
# FP64 pipe of a GB300: 152 SMs x 4 sub-partitions, one DFMA warp instruction
# (32 lanes x 2 flop) per 64 cycles per sub-partition = 608 flop per cycle
FP64_FLOP_PER_CYCLE = 152 * 4 * 32 * 2 // 64

# dram__bytes_read.sum + dram__bytes_write.sum of one block_update<64, double>
# launch (ncu, 4096x4096 graded, b = 32, every pair updated) divided by the
# (pair, row) units it processed: 477.9 MB / (64 pairs x 8192 rows).  The
# traffic grows in proportion to the units, so a launch's traffic is this
# figure times its units (algorithmic: 1024 B per unit, read + write).
UPDATE_BYTES_PER_PAIR_ROW = 477.94e6 / (64 * 8192)
# The same figure for update_split<64> (the tensor-core update, G and V in one
# launch): ncu, 4096x4096 graded, b = 32, every pair updated, 279.16 MB read +
# 209.30 MB written for 2 x 64 pairs x 4096 rows.
SPLIT_UPDATE_BYTES_PER_PAIR_ROW = 488.461e6 / (2 * 64 * 4096)
# bf16 digit products per FP64 product in the split contractions: the mma.sync
# Gram and update (contraction "split_sync") use 9 7-bit slices (levels
# i + l <= 8: 45 products), the tcgen05 Gram and update (the default "split")
# 8 8-bit slices (levels i + l <= 7: 36 products)
SPLIT_PRODUCTS = 45
TC_PRODUCTS = 36
# dram__bytes_read.sum + dram__bytes_write.sum of one update_tc<64> launch (ncu,
# 4096x4096 graded, b = 32, first sweep: every pair updated; 283.55 MB read +
# 207.89 MB written) divided by its 64 pairs x 8192 (G and V) rows
TC_UPDATE_BYTES_PER_PAIR_ROW = 491.436e6 / (64 * 8192)

WORKLOADS = {
    # name: (m, n, generator, description)
    "graded8192": (8192, 8192, "graded", "8192x8192 N(0,1), column j x 10^u_j, u_j~U(-4,0)"),
    "graded4096": (4096, 4096, "graded", "4096x4096 N(0,1), column j x 10^u_j, u_j~U(-4,0)"),
    "small512": (512, 256, "planted", "512x256 U diag(s) V^T, s geometric 1..1e-8, Haar U,V"),
    "hsvd4096": (4096, 4096, "hsvd", "HSVD of 4096x4096 N(0,1), J=diag(+1 x2048, -1 x2048)"),
    "mixed8192x4096": (8192, 4096, "mixed", "8192x4096 U diag(s) V^T, s_i=10^(-12 x_i), x~U(0,1), Haar U,V; "
                                            "FP32 sweeps then FP64 sweeps"),
    "mixed2048x1024": (2048, 1024, "mixed", "2048x1024 U diag(s) V^T, s_i=10^(-12 x_i), x~U(0,1), Haar U,V; "
                                            "FP32 sweeps then FP64 sweeps"),
}


def fp64_peak_tflops(sustained: bool) -> tuple[float, str]:
    """FP64 contraction peak: measured bf16 dense peak x nominal FP64/bf16 ratio."""
    try:
        pk = json.load(open(PEAKS_FILE))
        bf16 = pk["bf16_tflops_sustained" if sustained else "bf16_tflops"]
        return bf16 * NOMINAL_FP64_TF / NOMINAL_BF16_TF, (
            f"measured bf16 {'sustained' if sustained else 'burst'} {bf16} TF/s x nominal FP64/bf16 "
            f"{NOMINAL_FP64_TF}/{NOMINAL_BF16_TF}")
    except Exception:
        fb = 1700.0 if sustained else 1900.0
        return fb * NOMINAL_FP64_TF / NOMINAL_BF16_TF, "fallback bf16 x nominal FP64/bf16 ratio"


def bf16_peak_tflops(sustained: bool) -> tuple[float, str]:
    """Measured dense bf16 tensor peak of the GB300s."""
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        pk = json.load(open(PEAKS_FILE))
        return float(pk[key]), f"MEASURED_PEAKS.json {key} = {pk[key]} TF/s"
    except Exception:
        fb = 1700.0 if sustained else 1900.0
        return fb, f"fallback bf16 {'sustained' if sustained else 'burst'} {fb} TF/s"


def make_input(name: str, seed: int) -> np.ndarray:
    from paper_1401_2720_gb300 import inputs

    m, n, kind, _ = WORKLOADS[name]
    if kind == "graded":
        return inputs.graded_gaussian(m, n, seed)
    if kind == "hsvd":
        return inputs.gaussian(m, n, seed)
    if kind == "mixed":
        return inputs.workload_mixed(m, n, seed)[0]
    return inputs.planted(m, n, inputs.geometric(n, 1.0, 1e-8), seed)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def variant_name(inner_sweeps: int) -> str:
    if inner_sweeps <= 1:
        return "block-oriented (one inner sweep)"
    return f"full block (at most {inner_sweeps} inner sweeps)"


# Block sweeps the GPU solve of each workload performs (seed 0, default b and
# strategy, split contractions), measured on a GB300: the reference arm, which
# runs no GPU, extrapolates its timed p-steps by this count, the same count the
# GPU arm measures and uses for its own cpu_baseline.
MEASURED_SWEEPS = {"graded8192": 10, "graded4096": 9, "small512": 17, "hsvd4096": 11, "mixed8192x4096": 33,
                   "mixed2048x1024": 27}


def cpu_sample(A: np.ndarray, b: int, strategy: str, sweeps: float, nplus: int | None = None,
               inner_sweeps: int = 1, budget_s: float = 15.0):
    """Time the oracle's block-oriented method on the full-size input with all
    host cores (threads over the disjoint pivot pairs of each p-step; bitwise
    the same result as one thread): whole p-steps of the first sweep, as many as
    fit in about budget_s seconds (at least one), then scale to s/matrix by
    p-steps per sweep x `sweeps` (the GPU solve's measured sweep count)."""
    import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    m, n = A.shape
    nb = n // b
    tab = oracle.strategy_array(strategy, nb)
    inner = oracle.strategy_array(strategy, 2 * b)
    G = np.asfortranarray(A).copy(order="F")
    V = np.asfortranarray(np.eye(n))
    done = 0
    t0 = time.perf_counter()
    while done < nb - 1:
        G, V, _ = oracle.block_pstep(G, V, b, tab[done], inner, nplus=nplus, inner_sweeps=inner_sweeps,
                                     inplace=True)
        done += 1
        if time.perf_counter() - t0 >= budget_s * done / (done + 1):
            break
    measured = time.perf_counter() - t0
    oracle.set_threads(1)
    per_step = measured / done
    est = per_step * (nb - 1) * sweeps
    sample = (f"{done} of the {nb - 1} p-steps of sweep 1 ({done * (nb // 2)} pivot pairs) of the oracle's "
              f"{variant_name(inner_sweeps)} method (b={b}) on the full {m}x{n} input, {cores} threads, "
              f"{measured:.2f} s measured; scaled by {nb - 1} p-steps/sweep x {sweeps:g} sweeps")
    return {"value": est, "unit": "s/matrix", "cores": cores, "kind": "oracle", "sample": sample,
            "measured_s": measured, "measured_psteps": done, "extrapolated_s": est, "sweeps": sweeps}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A = make_input(args.workload, args.seed)
    nplus = A.shape[1] // 2 if WORKLOADS[args.workload][2] == "hsvd" else None
    sweeps = MEASURED_SWEEPS[args.workload]
    vals, last = [], None
    budget = args.cpu_budget / max(1, args.warmup + args.steps)
    for i in range(args.warmup + args.steps):
        last = cpu_sample(A, args.b, args.strategy, sweeps, nplus, args.inner_sweeps, budget_s=budget)
        if i >= args.warmup:
            vals.append(last["value"])
    value = statistics.median(vals)
    m, n, _, desc = WORKLOADS[args.workload]
    cpu = dict(last)
    cpu["value"] = value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/matrix",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "b": args.b, "strategy": args.strategy,
                   "variant": variant_name(args.inner_sweeps)},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "s/matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": ("the reference is the paper's method as the CPU oracle; value extrapolates the measured p-steps "
                 "(cpu_baseline.measured_s per step) to a whole solve, so ms_per_step x steps is not wall time"),
    }
    print(json.dumps(line), flush=True)


def run_ordering_study(args) -> None:
    """Sweeps and time of every block ordering (Sec. 3 p-strategies, and the
    dynamic norm-sorted ordering over rR) on the graded 8192^2 SVD and the
    4096^2 HSVD, b = 32, split contractions; one solve each after a warm-up
    solve, CUDA events on the solve's stream.  One JSON line per solve and a
    summary line with the time ratios to reverse R|| (the paper's Fig. 6.1
    reports the other static strategies 14-21 % slower than reverse R||,
    reverse C|| about equal)."""
    import torch

    from paper_1401_2720_gb300 import build_ext
    from paper_1401_2720_gb300 import jsvd as J

    build_ext.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    orders = [("rR", False), ("rC", False), ("R", False), ("C", False), ("modulus", False), ("rR", True)]
    summary = {}
    for wl in args.study_workloads.split(","):
        m, n, kind, desc = WORKLOADS[wl]
        A = torch.from_numpy(np.ascontiguousarray(make_input(wl, args.seed).T)).to(dev).t()
        res = {}
        for strat, dyn in orders:
            kw = dict(b=32, strategy=strat, dynamic_order=dyn, return_info=True, max_sweeps=args.max_sweeps)
            solve = (lambda: J.hsvd(A, n // 2, **kw)) if kind == "hsvd" else (lambda: J.svd(A, **kw))
            solve()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, S, _, info = solve()
            e1.record()
            torch.cuda.synchronize()
            name = strat + ("+dynamic" if dyn else "")
            res[name] = {"s": e0.elapsed_time(e1) / 1e3, "sweeps": info["sweeps"], "converged": info["converged"],
                         "proper_rotations": info["proper_rotations"], "pairs_updated": info["pairs_updated"]}
            print(json.dumps({"study": "orderings", "workload": desc, "ordering": name, **res[name]}), flush=True)
        base = res["rR"]["s"]
        summary[wl] = {k: {"time_ratio_vs_rR": v["s"] / base, "sweeps": v["sweeps"]} for k, v in res.items()}
    print(json.dumps({"study": "orderings", "summary": summary}), flush=True)


def run_batched(args) -> None:
    """Forward (one graph launch over all matrices) + backward (adjoint of
    L = sum w_i s_i + <C, U V^T>, cotangents formed once outside the timed
    region) of the 4096-matrix uneven batch."""
    import torch

    from paper_1401_2720_gb300 import build_ext, inputs
    from paper_1401_2720_gb300 import jsvd as J

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    build_ext.build()
    mats, sig, ws, Cs = inputs.workload_batch(args.batch, seed=args.seed)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    A = pk.pack(mats, dev)
    tuned = None
    if args.b in (8, 16, 32):
        b = args.b
    else:
        # autotuned block width per bucket of n, outside the timed region
        from paper_1401_2720_gb300 import autotune

        t0 = time.perf_counter()
        tuned = autotune.tune(mats)
        b = autotune.block_widths(pk.n, tuned)
        strat, strat_times = autotune.tune_strategy(mats, tuned)
        tune_s = time.perf_counter() - t0
    pre = dict(preprocess=True) if args.preprocess else {}
    if tuned is not None:
        pre["strategy"] = strat
    U, S, V, infos, rc = J.svd_batched_packed(pk, A, b=b, return_info=True, max_sweeps=args.max_sweeps, **pre)
    Us, Vs = pk.unpack_mn(U), pk.unpack_nn(V)
    dU = torch.cat([torch.from_numpy(C).to(dev).mm(v).t().reshape(-1) for C, v in zip(Cs, Vs)])
    dV = torch.cat([torch.from_numpy(C).to(dev).t().mm(u).t().reshape(-1) for C, u in zip(Cs, Us)])
    dS = torch.cat([torch.from_numpy(w).to(dev) for w in ws])
    for _ in range(args.warmup):
        U, S, V = J.svd_batched_packed(pk, A, b=b, max_sweeps=args.max_sweeps, **pre)
        J.svd_backward_packed(pk, U, S, V, dU, dS, dV)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    J.profile(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    clocks.start()
    fwd = bwd = 0.0
    for _ in range(args.steps):
        e[0].record(stream)
        U, S, V, infos, rc = J.svd_batched_packed(pk, A, b=b, return_info=True, max_sweeps=args.max_sweeps,
                                                  **pre)
        e[1].record(stream)
        dA = J.svd_backward_packed(pk, U, S, V, dU, dS, dV)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwd += e[0].elapsed_time(e[1])
        bwd += e[1].elapsed_time(e[2])
    clk = clocks.stop()
    prof = J.profile_read()
    J.profile(False)
    fwd /= args.steps
    bwd /= args.steps
    ms_step = fwd + bwd
    flops = prof["other"][2] / args.steps
    # accuracy spot check against the planted spectra (normwise per matrix)
    err = max(float(np.max(np.abs(s.cpu().numpy() - st)) / st[0]) for s, st in zip(pk.unpack_n(S), sig))
    # the plain form on the same matrices, one solve per matrix (single-matrix
    # entry point, default options), on a fixed sample: outside the timed region
    sample = list(range(0, len(mats), max(1, len(mats) // args.plain_sample)))[: args.plain_sample]
    dev_mats = [torch.from_numpy(np.ascontiguousarray(mats[i].T)).to(dev).t() for i in sample]
    for a in dev_mats[:8]:
        J.svd(a)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i, a in zip(sample, dev_mats):
        _, s_i, _ = J.svd(a)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1) / len(sample)
    sample_fwd_share = sum(mats[i].shape[0] * mats[i].shape[1] ** 2 for i in sample) / sum(
        a.shape[0] * a.shape[1] ** 2 for a in mats) * len(mats) / len(sample)
    line = {
        "metric": METRIC, "value": ms_step / 1e3 / len(pk), "unit": "s/matrix", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batch of {len(pk)} matrices, m~U{{16..512}}, n~U{{8..m}}, s log-uniform "
                               f"[1e-6,1] with gaps >= 1e-3, Haar U,V; forward + adjoint backward",
                   "b": (args.b if tuned is None else
                         {f"n in {autotune.BUCKETS[k]}": v for k, v in sorted(tuned.items())}),
                   "autotune_s": None if tuned is None else tune_s,
                   "strategy": None if tuned is None else {"chosen": strat, "sample_s": strat_times},
                   "qr_preprocessing": "matrices with m >= 2n: A P = Q [R; 0], the method on R^T"
                   if args.preprocess else None},
        "matrices_per_s": len(pk) / (ms_step / 1e3),
        "plain_form": {"matrices": len(sample), "ms_per_matrix": plain_ms,
                       "forward_matrices_per_s": 1e3 / plain_ms,
                       "batched_forward_matrices_per_s": len(pk) / (fwd / 1e3),
                       "note": "the same matrices solved one at a time through jsvd.svd (forward only); an evenly "
                               "spaced sample of the batch, whose m n^2 work is "
                               f"{sample_fwd_share:.2f}x the batch average"},
        "forward_ms": fwd, "backward_ms": bwd, "tflops": flops / (ms_step * 1e-3) / 1e12,
        "sweeps_max": max(i["sweeps"] for i in infos), "sweeps_mean": statistics.mean(i["sweeps"] for i in infos),
        "converged": all(i["converged"] for i in infos), "max_normwise_sigma_err_vs_planted": err,
        "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def mixed_side(args, dev) -> dict:
    """Mixed FP32 -> FP64 against plain FP64 on the 8192 x 4096 planted
    workload (sigma in [1e-12, 1]), one solve each after one untimed mixed
    solve, CUDA events around each; outside any timed region."""
    import torch

    from paper_1401_2720_gb300 import jsvd as J

    wl = "mixed8192x4096"
    m, n, _, desc = WORKLOADS[wl]
    A = torch.from_numpy(np.ascontiguousarray(make_input(wl, args.seed).T)).to(dev).t()
    out = [(torch.empty((n, m), dtype=torch.float64, device=dev).t(), torch.empty(n, dtype=torch.float64, device=dev),
            torch.empty((n, n), dtype=torch.float64, device=dev).t()) for _ in range(2)]
    kw = dict(b=args.b, strategy=args.strategy, contraction=args.contraction)
    stream = torch.cuda.current_stream()
    J.svd(A, out=out[0], precision="mixed", max_sweeps=args.max_sweeps, **kw)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    _, _, _, inf_mx = J.svd(A, out=out[0], precision="mixed", max_sweeps=args.max_sweeps, return_info=True, **kw)
    ev[1].record(stream)
    ev[2].record(stream)
    _, _, _, inf_64 = J.svd(A, out=out[1], max_sweeps=max(args.max_sweeps, 60), return_info=True, **kw)
    ev[3].record(stream)
    torch.cuda.synchronize()
    t_mx, t_64 = ev[0].elapsed_time(ev[1]) / 1e3, ev[2].elapsed_time(ev[3]) / 1e3
    smx, s64 = out[0][1].cpu().numpy(), out[1][1].cpu().numpy()
    s_true = np.sort(10.0 ** (-12.0 * np.random.default_rng(args.seed).uniform(0.0, 1.0, size=n)))[::-1]
    return {"workload": desc, "mixed_s": t_mx, "plain_fp64_s": t_64, "speedup": t_64 / t_mx,
            "mixed_sweeps_fp32": inf_mx["sweeps_low"], "mixed_sweeps_fp64": inf_mx["sweeps"],
            "plain_sweeps": inf_64["sweeps"], "converged": bool(inf_mx["converged"] and inf_64["converged"]),
            "normwise_mixed_vs_planted": float(np.max(np.abs(smx - s_true)) / s_true[0]),
            "normwise_plain_vs_planted": float(np.max(np.abs(s64 - s_true)) / s_true[0]),
            "normwise_mixed_vs_plain": float(np.max(np.abs(smx - s64)) / s64[0]),
            "note": "measured after the timed region, CUDA events around one solve each"}


def run_gpu(args) -> None:
    import torch
    import torch.distributed as dist

    from paper_1401_2720_gb300 import build_ext, replicas
    from paper_1401_2720_gb300 import jsvd as J

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if rank == 0 or world == 1:
        build_ext.build()
    if world > 1:
        dist.barrier()

    m, n, _, desc = WORKLOADS[args.workload]
    A_host = make_input(args.workload, replicas.rank_seed(args.seed, rank))
    A = torch.from_numpy(np.ascontiguousarray(A_host.T)).to(dev).t()      # column-major view
    U = torch.empty((n, m), dtype=torch.float64, device=dev).t()
    S = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    kind = WORKLOADS[args.workload][2]
    kw = dict(b=args.b, strategy=args.strategy, max_sweeps=args.max_sweeps, inner_sweeps=args.inner_sweeps,
              contraction=args.contraction)
    if kind == "mixed":
        kw["precision"] = "mixed"

    def solve(Ain):
        if kind == "hsvd":
            return J.hsvd(Ain, n // 2, out=(U, S, V), return_info=True, **kw)
        return J.svd(Ain, out=(U, S, V), return_info=True, **kw)

    infos = []
    for _ in range(args.warmup):
        solve(A)
    torch.cuda.synchronize()

    # FP64 peak of this GPU, measured now (warm clocks), for the roofline
    peak_dfma, peak_dmma = J.fp64_peak(seconds=args.peak_seconds)
    peak_mma = J.bf16_mma_peak(seconds=args.peak_seconds) if args.contraction in ("split", "split_sync") else None
    torch.cuda.synchronize()

    # ---- timed region: K complete SVDs with inputs resident in HBM ------------
    stream = torch.cuda.current_stream()
    J.profile(True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, _, _, inf = solve(A)
        infos.append(inf)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    prof = J.profile_read()
    J.profile(False)
    ms_step, matrices = replicas.whole_job(ms_total / args.steps, 1, device=dev)
    value = replicas.seconds_per_matrix(ms_step, matrices)   # s per matrix, whole job

    # ---- e2e: host (pinned) -> device, SVD, results -> host --------------------
    e2e = None
    if not args.no_e2e:
        A_pin = torch.from_numpy(np.ascontiguousarray(A_host.T)).pin_memory()
        U_h = torch.empty((n, m), dtype=torch.float64).pin_memory()
        S_h = torch.empty(n, dtype=torch.float64).pin_memory()
        V_h = torch.empty((n, n), dtype=torch.float64).pin_memory()
        A_dev = torch.empty((n, m), dtype=torch.float64, device=dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            A_dev.copy_(A_pin, non_blocking=True)
            solve(A_dev.t())
            U_h.copy_(U.t(), non_blocking=True)
            S_h.copy_(S, non_blocking=True)
            V_h.copy_(V.t(), non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms, e2e_mats = replicas.whole_job(f0.elapsed_time(f1) / args.e2e_steps, 1, device=dev)
        e2e = {"value": replicas.seconds_per_matrix(e2e_ms, e2e_mats), "unit": "s/matrix",
               "h2d_bytes_per_step": m * n * 8 * world,
               "d2h_bytes_per_step": (m * n + n + n * n) * 8 * world}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ---------------------------------------
    flops_total = sum(v[2] for v in prof.values())
    dom = max(("gram", "jacobi", "update"), key=lambda c: prof[c][0])
    last_b = infos[-1]["b"]
    d_ms, d_launch, d_flops = prof[dom]
    derived, derived_src = fp64_peak_tflops(sustained=True)
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    peak = FP64_FLOP_PER_CYCLE * sm_mhz * 1e6 / 1e12
    achieved = d_flops / (d_ms * 1e-3) / 1e12 if d_ms > 0 else 0.0
    traffic = None
    bb = 2 * last_b
    per_row = {"split": TC_UPDATE_BYTES_PER_PAIR_ROW, "split_sync": SPLIT_UPDATE_BYTES_PER_PAIR_ROW,
               "fp64": UPDATE_BYTES_PER_PAIR_ROW}[args.contraction]
    if dom == "update" and d_launch and per_row is not None:
        # ncu DRAM bytes per (pair, row) of the update kernel x the launch's units
        traffic = per_row * (d_flops / (2.0 * bb * bb)) / d_launch
    fp64_src = (f"FP64 pipe: {FP64_FLOP_PER_CYCLE} flop/cycle (152 SMs x 4 sub-partitions x one DFMA warp "
                f"instruction per 64 cycles, the sm__inst_executed_pipe_fp64 peak) x median SM clock "
                f"{sm_mhz:.0f} MHz in the timed region; in-run probes: DMMA {peak_dmma:.3f}, DFMA "
                f"{peak_dfma:.3f} TFLOP/s")
    if args.contraction in ("split", "split_sync") and dom in ("gram", "update"):
        # tensor-core kernels: each FP64 product is `products` bf16 digit products
        products = TC_PRODUCTS if args.contraction == "split" else SPLIT_PRODUCTS
        bf16_peak, bf16_src = bf16_peak_tflops(sustained=True)
        tensor = products * achieved
        roofline = {"bound": "tensor", "achieved": tensor, "peak": bf16_peak, "unit": "TFLOP/s",
                    "frac": tensor / bf16_peak, "traffic": traffic,
                    "kernel": ({"gram": "gram_tc", "update": "update_tc"} if args.contraction == "split"
                               else {"gram": "gram_split", "update": "update_split"})[dom],
                    "launches": d_launch,
                    "peak_source": bf16_src + " (of measured); achieved = "
                                   f"{products} bf16 digit products x the kernel's algorithmic FP64 flops / "
                                   "its CUDA-event time",
                    "fp64_equivalent_tflops": achieved,
                    "mma_sync_bf16_peak": peak_mma,
                    "frac_of_mma_sync_peak": tensor / peak_mma if peak_mma else None}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if peak else None, "traffic": traffic,
                    "kernel": {"gram": "gram_partial", "jacobi": "pair_jacobi", "update": "block_update"}[dom],
                    "launches": d_launch, "peak_source": fp64_src,
                    "peak_derived": {"value": derived, "source": derived_src}}
    kernels = {c: {"ms": prof[c][0], "launches": prof[c][1], "tflops": (prof[c][2] / (prof[c][0] * 1e-3) / 1e12)
                   if prof[c][0] > 0 else None, "share": prof[c][0] / ms_total if ms_total else None}
               for c in ("gram", "jacobi", "update", "update_v")}
    if args.contraction in ("split", "split_sync"):
        kernels["update"]["note"] = ("update of G and V in one launch (tcgen05, 8-bit digits)" if args.contraction ==
                                     "split" else "update of G and V in one launch (mma.sync, 7-bit digits)")
        kernels["gram"]["note"] = ("Gram partials on tcgen05 (8-bit digits)" if args.contraction == "split"
                                   else "Gram partials on mma.sync (7-bit digits)")
        for c in ("gram", "update"):
            if kernels[c]["tflops"]:
                pr = TC_PRODUCTS if args.contraction == "split" else SPLIT_PRODUCTS
                kernels[c]["tensor_tflops"] = pr * kernels[c]["tflops"]
        kernels["update_v"]["note"] = "no side-stream V update with split contractions"
    else:
        kernels["update_v"]["note"] = ("V update on the low-priority side stream: it runs in the main stream's "
                                       "gaps, so its event time includes waiting for SMs and overlaps the other "
                                       "classes")

    cpu = None
    mixed_report = None
    if kind == "mixed" and not args.no_compare:
        # plain FP64 run of the same matrix, outside the timed region
        kw64 = dict(kw)
        kw64.pop("precision")
        kw64["max_sweeps"] = max(args.max_sweeps, 60)   # let the plain FP64 solve converge
        U64 = torch.empty_like(U)
        S64 = torch.empty_like(S)
        V64 = torch.empty_like(V)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        _, _, _, inf64 = J.svd(A, out=(U64, S64, V64), return_info=True, **kw64)
        g1.record(stream)
        torch.cuda.synchronize()
        s64 = S64.cpu().numpy()
        smx = S.cpu().numpy()
        rel = np.abs(smx - s64) / s64
        s_true = np.sort(10.0 ** (-12.0 * np.random.default_rng(args.seed).uniform(0.0, 1.0, size=n)))[::-1]
        mixed_report = {
            "plain_fp64_s": g0.elapsed_time(g1) / 1e3, "mixed_s": ms_step / 1e3,
            "speedup": (g0.elapsed_time(g1) / 1e3) / (ms_step / 1e3),
            "plain_sweeps": inf64["sweeps"], "mixed_sweeps_fp32": infos[-1]["sweeps_low"],
            "mixed_sweeps_fp64": infos[-1]["sweeps"],
            "normwise_vs_plain": float(np.max(np.abs(smx - s64)) / s64[0]),
            "max_rel_vs_plain": float(rel.max()),
            "rel_vs_plain_by_decade": {f"1e{-d}..1e{-d-1}": float(rel[(s64 <= 10.0 ** -d) & (s64 > 10.0 ** (-d - 1))].max())
                                       for d in range(0, 12) if np.any((s64 <= 10.0 ** -d) & (s64 > 10.0 ** (-d - 1)))},
            "normwise_mixed_vs_planted": float(np.max(np.abs(smx - s_true)) / s_true[0]),
            "normwise_plain_vs_planted": float(np.max(np.abs(s64 - s_true)) / s_true[0]),
            "orth_V_mixed": float((V.t() @ V - torch.eye(n, device=dev, dtype=torch.float64)).abs().max()),
        }

    cpu = None
    if world == 1 and not args.no_cpu:
        sweeps = statistics.mean(i["sweeps"] for i in infos)
        if mixed_report:
            sweeps = mixed_report["plain_sweeps"]
        cpu = cpu_sample(A_host, args.b if args.b else infos[-1]["b"], args.strategy, sweeps,
                         n // 2 if kind == "hsvd" else None, args.inner_sweeps, budget_s=args.cpu_budget)

    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "s/matrix", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "seed": args.seed, "b": last["b"], "strategy": args.strategy,
                   "variant": variant_name(args.inner_sweeps), "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tflops": flops_total / (ms_total * 1e-3) / 1e12 if ms_total else None,
        "sweeps": [i["sweeps"] for i in infos], "converged": all(i["converged"] for i in infos),
        "roofline": roofline, "kernels": kernels,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "clocks": clk,
    }
    if mixed_report:
        line["mixed_vs_plain"] = mixed_report
    elif world == 1 and args.workload == "graded8192" and not args.no_mixed:
        line["mixed_vs_plain"] = mixed_side(args, dev)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="graded8192", choices=sorted(WORKLOADS) + ["batched4096"])
    p.add_argument("--batch", type=int, default=4096)
    p.add_argument("--plain-sample", type=int, default=256,
                   help="batched workload: matrices solved one at a time for the plain-form comparison")
    p.add_argument("--b", type=int, default=None,
                   help="block width (default 32; the batched workload autotunes it per bucket of n)")
    p.add_argument("--strategy", default=None, help="pivot strategy (default rR; modulus for small512)")
    p.add_argument("--max-sweeps", type=int, default=30)
    p.add_argument("--contraction", default="split", choices=["fp64", "split", "split_sync"],
                   help="FP64 block contractions: FP64 FMA kernels, or split bf16 digits on the tensor cores "
                        "(split: tcgen05 Gram and update; split_sync: mma.sync Gram and update)")
    p.add_argument("--inner-sweeps", type=int, default=1,
                   help="inner sweeps per pivot pair: 1 = block-oriented, 30 = full block (Sec. 4.3)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--preprocess", action="store_true",
                   help="batched workload: QR preprocessing (column pivoting) of the matrices with m >= 2n")
    p.add_argument("--study", default=None, choices=["orderings"],
                   help="instead of the benchmark line: the block-ordering study")
    p.add_argument("--study-workloads", default="graded8192,hsvd4096")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-compare", action="store_true")
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the mixed-vs-plain side measurement (8192 x 4096) of the default workload")
    p.add_argument("--cpu-budget", type=float, default=15.0,
                   help="seconds of oracle time (all host cores) per CPU-baseline measurement")
    p.add_argument("--peak-seconds", type=float, default=2.0)
    args = p.parse_args()
    if args.b is None and args.workload != "batched4096":
        # block widths chosen by timing b in {8, 16, 32} on this GPU (split
        # contractions): 32 for the graded 8192^2, HSVD 4096^2 and mixed
        # workloads; 16 for the 512 x 256 one (the width its configuration names)
        args.b = 16 if args.workload == "small512" else 32
    if args.strategy is None:
        args.strategy = "modulus" if args.workload == "small512" else "rR"
    if args.study == "orderings":
        run_ordering_study(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched4096":
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
