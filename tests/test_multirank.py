"""The multi-rank aggregation of bench.py (replicas, one problem per rank) on
CPU with the gloo backend, world size 2: the job time is the slowest rank's,
the units are summed over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist, torch.device("cpu"))
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    for _, ms, units in out:
        assert ms == 15.0 and units == 300.0


def test_aggregate_single_rank():
    import torch
    import bench
    assert bench.aggregate(7.0, 3.0, None, torch.device("cpu")) == (7.0, 3.0)
