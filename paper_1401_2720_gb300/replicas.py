"""Multi-GPU runs are replicas: every rank solves its own matrices on its own
GPU and nothing is exchanged on the data path (the method's multi-GPU level is
not part of this library).  Only the timing is combined across ranks."""

from __future__ import annotations

import torch
import torch.distributed as dist


def rank_seed(base_seed: int, rank: int) -> int:
    """Each rank draws an independent matrix: seed base + rank."""
    return int(base_seed) + int(rank)


def whole_job(ms_local: float, matrices_local: int, device=None) -> tuple[float, int]:
    """(max over ranks of the step time in ms, total matrices of all ranks).
    Without an initialized process group this is the local pair."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), int(matrices_local)
    dev = torch.device("cpu") if device is None else torch.device(device)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    c = torch.tensor([int(matrices_local)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def seconds_per_matrix(ms_max: float, total_matrices: int) -> float:
    """Whole-job s/matrix: the slowest rank's time over all matrices solved."""
    return ms_max / 1e3 / max(total_matrices, 1)
