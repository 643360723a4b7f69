"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
independent alignment (weak scaling, no data-path collective); the job's time
is the slowest rank's and its units are the sum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.reduce_over_ranks([12.5, 30.0][rank], [1000.0, 3000.0][rank], world, device="cpu")
    a, starts = bench.workload(bench.WORKLOADS["pt128"], rank)
    out.put((rank, ms, units, int(a.codes[:, :50].sum()), int(starts[0].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in res:
        assert r[1] == 30.0 and r[2] == 4000.0
    assert res[0][3:] != res[1][3:]  # each rank has its own alignment and starts
