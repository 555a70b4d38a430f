"""Multi-rank host logic on CPU with gloo, world size 2: walker sharding and
the max-over-ranks timing reduction used by bench.py (replicas only; no
collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1204_1121_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import blip_inputs as bi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # strong scaling: ranges partition the walkers
        w0, w1 = replicas.walker_range(10, rank, world)
        rngs = [None] * world
        dist.all_gather_object(rngs, (w0, w1))
        # weak scaling: each rank's positions differ
        w = bi.workload("tio2_batch", batch=4, n_walkers=2)
        w.pos_seed = replicas.weak_seed(w.pos_seed, rank)
        pos, _ = w.positions()
        firsts = [None] * world
        dist.all_gather_object(firsts, pos[0].tolist())
        # timing reduction: max over ranks
        m = replicas.max_over_ranks(1.5 + rank)
        out[rank] = (rngs, firsts, m)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_max_reduction():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    rngs, firsts, m = out[0]
    assert rngs == [(0, 5), (5, 10)]
    assert firsts[0] != firsts[1]
    assert m == 2.5 and out[1][2] == 2.5


def test_walker_range_partitions():
    for W in (0, 1, 7, 256):
        for N in (1, 2, 3, 8):
            seen = []
            for r in range(N):
                a, b = replicas.walker_range(W, r, N)
                seen.extend(range(a, b))
            assert seen == list(range(W))
    with pytest.raises(ValueError):
        replicas.walker_range(4, 2, 2)


def test_max_over_ranks_single_process():
    assert replicas.max_over_ranks(3.25) == 3.25
