"""The multi-GPU benchmark path runs independent replicas (one per rank, no collective on
the data path); its host logic -- the barrier and the max-over-ranks of the timed region --
is exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
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
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        ms = [12.0, 15.0][rank]  # the slower rank decides the job time
        m = bench.max_over_ranks(dist, ms)
        out[rank] = bench.aggregate_rate(1000, 10, m, world)
        out[world + rank] = m
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", 2 * world)
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[world] == out[world + 1] == 15.0
    # 2 ranks x 1000 units x 10 steps in 15 ms
    assert out[0] == out[1] == pytest.approx(2 * 1000 * 10 / 0.015)
