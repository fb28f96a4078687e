"""The bench's multi-rank logic on CPU: world size 2 over gloo, replicas with no
data-path collective, the job time is the slowest rank's, the rate counts all replicas."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(torch, 1.0 + rank, "cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.0
    import bench
    assert bench.aggregate_rate(2, 128000, 10, 2.0) == pytest.approx(2 * 128000 * 10 / 2.0)
    assert bench.max_over_ranks(torch, 3.5, "cpu") == 3.5      # single process: unchanged
