"""The multi-rank (replica) path on CPU with the gloo backend, world size 2:
the whole-job time is the slowest rank's, the matrices add up, and ranks draw
independent inputs."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1401_2720_gb300 import inputs, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, count = replicas.whole_job(100.0 * (rank + 1), 1 + rank)
        a = inputs.graded_gaussian(8, 4, replicas.rank_seed(7, rank))
        gathered = [None] * world
        dist.all_gather_object(gathered, float(a[0, 0]))
        out.put((rank, ms, count, gathered))
    finally:
        dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, count, gathered in res:
        assert ms == 200.0 and count == 3
        assert gathered[0] != gathered[1]            # independent inputs per rank
    assert replicas.seconds_per_matrix(200.0, 3) == pytest.approx(0.2 / 3)


def test_single_process_is_local():
    assert replicas.whole_job(12.5, 4) == (12.5, 4)
