"""The replica path of bench.py (N > 1): two gloo ranks on CPU aggregate
their timings as the slowest rank's time and the sum of their units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.aggregate_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist)
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 300.0)


def test_single_process_is_unchanged():
    import bench
    assert bench.aggregate_ranks(3.5, 7.0, None) == (3.5, 7.0)
