"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own
replica workload (every source, tag = rank); the timing is the max over
ranks and the units the sum, with no data exchanged otherwise."""
import os
import socket

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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b, tag = bench.rank_workload(1000, rank, world)
    T, units = bench.reduce_over_ranks(1.0 + rank, [10.0 * (rank + 1), 3.0], world, dist)
    q.put((rank, a, b, tag, T, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, a, b, tag, T, units in out:
        assert (a, b) == (0, 1000)  # each replica covers every source
        assert tag == rank          # independent walks per rank
        assert T == 2.0             # max over ranks
        assert units == [30.0, 6.0]  # units summed over ranks
