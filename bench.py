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

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel from an ncu capture of the current kernel build (None until taken).
TRAFFIC_PER_LAUNCH: dict = {}

WORKLOADS = {
    # name: (m, n, generator, description)
    "graded8192": (8192, 8192, "graded", "8192x8192 N(0,1), column j x 10^u_j, u_j~U(-4,0)"),
    "graded4096": (4096, 4096, "graded", "4096x4096 N(0,1), column j x 10^u_j, u_j~U(-4,0)"),
    "small512": (512, 256, "planted", "512x256 U diag(s) V^T, s geometric 1..1e-8, Haar U,V"),
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


def make_input(name: str, seed: int) -> np.ndarray:
    from paper_1401_2720_gb300 import inputs

    m, n, kind, _ = WORKLOADS[name]
    if kind == "graded":
        return inputs.graded_gaussian(m, n, seed)
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


def cpu_sample(A: np.ndarray, b: int, strategy: str, pairs: int, sweeps_hint: float):
    """Time the oracle's block-oriented p-step on `pairs` pivot pairs of the
    full-size input and scale to s/matrix: (t / pairs) x pairs per sweep x sweeps."""
    import oracle

    m, n = A.shape
    nb = n // b
    tab = oracle.strategy_array(strategy, nb)
    inner = oracle.strategy_array(strategy, 2 * b)
    G = np.asfortranarray(A)
    V = np.asfortranarray(np.eye(n))
    step = tab[0][:pairs]
    t0 = time.perf_counter()
    oracle.block_pstep(G, V, b, step, inner)
    t = time.perf_counter() - t0
    per_pair = t / len(step)
    pairs_per_sweep = (nb // 2) * (nb - 1)
    est = per_pair * pairs_per_sweep * sweeps_hint
    sample = (f"{len(step)} pivot pairs of p-step 1 of the oracle's block-oriented method (b={b}) on the "
              f"full {m}x{n} input, {t:.2f} s, scaled by {pairs_per_sweep} pairs/sweep x {sweeps_hint:g} sweeps")
    return est, sample


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A = make_input(args.workload, args.seed)
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample = cpu_sample(A, args.b, args.strategy, args.cpu_pairs, args.cpu_sweeps)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    m, n, _, desc = WORKLOADS[args.workload]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/matrix",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "b": args.b, "strategy": args.strategy},
        "cpu_baseline": {"value": value, "unit": "s/matrix", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "s/matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args) -> None:
    import torch
    import torch.distributed as dist

    from paper_1401_2720_gb300 import build_ext
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
    A_host = make_input(args.workload, args.seed + rank)
    A = torch.from_numpy(np.ascontiguousarray(A_host.T)).to(dev).t()      # column-major view
    U = torch.empty((n, m), dtype=torch.float64, device=dev).t()
    S = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    kw = dict(b=args.b, strategy=args.strategy, max_sweeps=args.max_sweeps)

    infos = []
    for _ in range(args.warmup):
        _, _, _, inf = J.svd(A, out=(U, S, V), return_info=True, **kw)
    torch.cuda.synchronize()

    # FP64 peak of this GPU, measured now (warm clocks), for the roofline
    peak_dfma, peak_dmma = J.fp64_peak(seconds=args.peak_seconds)
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
        _, _, _, inf = J.svd(A, out=(U, S, V), return_info=True, **kw)
        infos.append(inf)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    prof = J.profile_read()
    J.profile(False)
    ms_step = ms_total / args.steps
    if world > 1:
        t = torch.tensor([ms_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = ms_step / 1e3 / world                    # s per matrix, whole job

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
            J.svd(A_dev.t(), out=(U, S, V), **kw)
            U_h.copy_(U.t(), non_blocking=True)
            S_h.copy_(S, non_blocking=True)
            V_h.copy_(V.t(), non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1) / args.e2e_steps
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": e2e_ms / 1e3 / world, "unit": "s/matrix", "h2d_bytes_per_step": m * n * 8 * world,
               "d2h_bytes_per_step": (m * n + n + n * n) * 8 * world}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ---------------------------------------
    flops_total = sum(v[2] for v in prof.values())
    dom = max(("gram", "jacobi", "update"), key=lambda c: prof[c][0])
    d_ms, d_launch, d_flops = prof[dom]
    derived, derived_src = fp64_peak_tflops(sustained=True)
    peak = max(peak_dmma, peak_dfma)
    achieved = d_flops / (d_ms * 1e-3) / 1e12 if d_ms > 0 else 0.0
    traffic = TRAFFIC_PER_LAUNCH.get((args.workload, dom))
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": traffic,
                "kernel": {"gram": "gram_partial", "jacobi": "pair_jacobi", "update": "block_update"}[dom],
                "launches": d_launch,
                "peak_source": (f"FP64 peak measured in this run by the library's probe: mma.sync m8n8k4 "
                                f"{peak_dmma:.3f}, DFMA {peak_dfma:.3f} TFLOP/s (of measured)"),
                "peak_derived": {"value": derived, "source": derived_src}}
    kernels = {c: {"ms": prof[c][0], "launches": prof[c][1], "tflops": (prof[c][2] / (prof[c][0] * 1e-3) / 1e12)
                   if prof[c][0] > 0 else None, "share": prof[c][0] / ms_total if ms_total else None}
               for c in ("gram", "jacobi", "update")}

    cpu = None
    if world == 1 and not args.no_cpu:
        sweeps = statistics.mean(i["sweeps"] for i in infos)
        est, sample = cpu_sample(A_host, args.b if args.b else infos[-1]["b"], args.strategy,
                                 args.cpu_pairs, sweeps)
        cpu = {"value": est, "unit": "s/matrix", "cores": 1, "kind": "oracle", "sample": sample}

    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "s/matrix", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "seed": args.seed, "b": last["b"], "strategy": args.strategy,
                   "variant": "block-oriented (one inner sweep)", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tflops": flops_total / (ms_total * 1e-3) / 1e12 if ms_total else None,
        "sweeps": [i["sweeps"] for i in infos], "converged": all(i["converged"] for i in infos),
        "roofline": roofline, "kernels": kernels,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="graded8192", choices=sorted(WORKLOADS))
    p.add_argument("--b", type=int, default=32)
    p.add_argument("--strategy", default="rR")
    p.add_argument("--max-sweeps", type=int, default=30)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-pairs", type=int, default=32)
    p.add_argument("--peak-seconds", type=float, default=2.0)
    p.add_argument("--cpu-sweeps", type=float, default=12.0,
                   help="sweep count the reference arm scales its sample by")
    args = p.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
