"""The multi-GPU benchmark path: the single-mesh workload runs independent replicas (one per
rank), the batched workloads split their instances over the ranks; neither has a collective
on the data path.  The host logic -- the barrier, the max-over-ranks of the timed region,
the instance partition and the DOF sum -- is exercised here with two gloo ranks on the CPU."""
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


def _partition_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    from paper_1904_11147_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for k, w_all in enumerate((W.burgers_2d_batched(), W.euler_2d_batched())):
            cells = [a * b for a, b in zip(w_all.nx, w_all.ny)]
            mine = bench.partition_instances(cells, world)[rank]
            w = bench.subset_workload(w_all, mine)
            dofs = w.cells * w.nvars * w.nmodes
            total = bench.sum_over_ranks(dist, float(dofs))
            got = [None] * world
            dist.all_gather_object(got, mine)
            seen = sorted(i for part in got for i in part)
            ok_once = seen == list(range(w_all.n_inst))
            loads = [sum(cells[i] for i in part) for part in got]
            ok_bal = max(loads) - sum(loads) / world < max(cells)
            ok_dofs = total == w_all.cells * w_all.nvars * w_all.nmodes
            ok_params = all(w.params[j] == w_all.params[i] and w.nx[j] == w_all.nx[i] for j, i in enumerate(mine))
            out[4 * k + rank] = float(ok_once and ok_bal and ok_dofs and ok_params)
            out[4 * k + 2 + rank] = max(loads) / (sum(loads) / world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_batched_instances():
    """The batched workloads are split over the ranks (largest instance first, to the least
    loaded rank): every instance lands on exactly one rank with its own parameters, no rank
    carries more than the mean load plus one instance, and the ranks' DOF counts add up
    to the whole batch's."""
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", 8)
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert list(out[0:2]) == [1.0, 1.0] and list(out[4:6]) == [1.0, 1.0]
    # the imbalance of these two batches is small in practice
    assert out[2] < 1.02 and out[6] < 1.02, (out[2], out[6])
