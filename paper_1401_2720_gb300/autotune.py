"""Block-width and pivot-schedule autotuner for the batched solver.

The block width b trades the work of the inner Jacobi sweep (grows with b)
and the number of p-steps and launches per sweep (shrinks with b) against the
number of block sweeps the method needs, which depends on the matrices.  Per
bucket of column counts n, `tune` times one batched solve of a sample of the
bucket's matrices for each candidate b and keeps the fastest.  The table is
kept per device name for the life of the process (and in a JSON file when
`path` is given).  `tune_strategy` then picks the pivot strategy (the
p-strategy of Sec. 3 every matrix of the batch uses) by timing a sample of
the whole batch, with the tuned widths, for each candidate strategy.
"""

from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import jsvd as J

BUCKETS = ((1, 32), (33, 64), (65, 128), (129, 256), (257, 512), (513, 1024))
_cache: dict[str, dict[int, int]] = {}


def bucket_of(n: int) -> int:
    for k, (lo, hi) in enumerate(BUCKETS):
        if lo <= n <= hi:
            return k
    raise ValueError(f"n = {n} is outside the tuned range")


def _time_batch(mats, b, device, repeats: int, strategy: str = "rR") -> float:
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    A = pk.pack(mats, device)
    J.svd_batched_packed(pk, A, b=b, strategy=strategy)   # warm-up (also builds the tables)
    torch.cuda.synchronize(device)
    best = float("inf")
    for _ in range(repeats):
        t0 = time.perf_counter()
        J.svd_batched_packed(pk, A, b=b, strategy=strategy)
        torch.cuda.synchronize(device)
        best = min(best, time.perf_counter() - t0)
    return best


def tune(mats, candidates=(8, 16, 32), sample: int = 64, repeats: int = 3, seed: int = 0,
         path: str | None = None, device=None) -> dict[int, int]:
    """{bucket index: fastest b} for the buckets that `mats` populate."""
    device = torch.device(device or "cuda")
    name = torch.cuda.get_device_name(device)
    table = dict(_cache.get(name, {}))
    if path and os.path.exists(path):
        table.update({int(k): v for k, v in json.load(open(path)).get(name, {}).items()})
    rng = np.random.default_rng(seed)
    by_bucket: dict[int, list] = {}
    for a in mats:
        by_bucket.setdefault(bucket_of(a.shape[1]), []).append(a)
    for k, group in sorted(by_bucket.items()):
        if k in table:
            continue
        pick = [group[i] for i in rng.choice(len(group), size=min(sample, len(group)), replace=False)]
        times = {b: _time_batch(pick, b, device, repeats) for b in candidates}
        # the largest width within 5 % of the fastest: in the whole batch a
        # larger b also means fewer lock-step p-steps per sweep, which a
        # bucket timed alone does not see
        fastest = min(times.values())
        table[k] = max(b for b, t in times.items() if t <= 1.05 * fastest)
    _cache[name] = table
    if path:
        data = json.load(open(path)) if os.path.exists(path) else {}
        data[name] = {str(k): v for k, v in table.items()}
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
    return table


def block_widths(ns, table: dict[int, int], default: int = 8) -> np.ndarray:
    """Per-matrix b from a tuned table (default for untuned buckets)."""
    return np.array([table.get(bucket_of(int(n)), default) for n in ns], dtype=np.int32)


_strategy_cache: dict[str, str] = {}


def tune_strategy(mats, table: dict[int, int], candidates=("rR", "rC", "modulus"), sample: int = 128,
                  repeats: int = 2, seed: int = 0, device=None) -> tuple[str, dict[str, float]]:
    """(fastest strategy, {strategy: seconds}) for a random sample of the
    batch solved with the tuned block widths."""
    device = torch.device(device or "cuda")
    rng = np.random.default_rng(seed)
    pick = [mats[i] for i in rng.choice(len(mats), size=min(sample, len(mats)), replace=False)]
    b = block_widths([a.shape[1] for a in pick], table)
    times = {s: _time_batch(pick, b, device, repeats, strategy=s) for s in candidates}
    best = min(times, key=times.get)
    _strategy_cache[torch.cuda.get_device_name(device)] = best
    return best, times
