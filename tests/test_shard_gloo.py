"""Host-side logic of the multi-GPU batch path, run as two gloo ranks on CPU:
every rank derives its shard of the independent instances from the sizes
alone (no data exchange on the data path), the shards are disjoint, cover
the batch and balance the work estimate; the ranks agree on the max-over-ranks
step time the benchmark reports."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, count, out):
    import torch
    import torch.distributed as dist

    from paper_2508_04370_gb300.batch import instance_cost, shard_sizes

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = synth.batched_sizes(count=count, seed=3)
    mine = shard_sizes(sizes, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    load = torch.tensor([sum(instance_cost(*sizes[i], 5 * sizes[i][1]) for i in mine)], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    # the bench's max over ranks of the per-rank step time
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (got, [float(x) for x in loads], float(t))
    dist.destroy_process_group()


@pytest.mark.parametrize("count", [64, 257])
def test_batch_shards_two_ranks(count):
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, count, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    got0, loads, tmax = out[0]
    assert out[1][0] == got0  # both ranks see the same partition
    ids = sorted(i for part in got0 for i in part)
    assert ids == list(range(count))  # disjoint and complete
    assert max(loads) <= 1.02 * min(loads)  # LPT balance on the work estimate
    assert tmax == 2.0 and out[1][2] == 2.0
