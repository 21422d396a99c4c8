"""World-size-2 gloo test of the multi-GPU host logic on CPU: instance
sharding, max-over-ranks timing and the gather of per-instance scalars."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2410_02532_gb300 import shard


def test_shard_partitions_exactly():
    for total in (0, 1, 7, 15, 256):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s = shard.shard(total, world, r)
                seen.extend(s)
                assert len(s) in (total // world, total // world + 1)
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(shard.shard(10, world, rank))
        t = shard.max_over_ranks(1.5 + rank, dist)
        g = shard.gather_to_rank0({"rank": rank, "instances": mine, "power": [0.1 * i for i in mine]},
                                  dist)
        dist.barrier()
        q.put((rank, t, g))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        rank, t, g = q.get(timeout=120)
        out[rank] = (t, g)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.5
    g = out[0][1]
    assert out[1][1] is None
    assert [x["rank"] for x in g] == [0, 1]
    assert sorted(i for x in g for i in x["instances"]) == list(range(10))


def test_single_process_fallbacks():
    assert shard.max_over_ranks(3.0) == 3.0
    assert shard.gather_to_rank0(5) == [5]
    _ = torch
