"""Host logic of the multi-rank benchmark path: the batch instances are
independent lattices, so ranks split them (no data-path collective) and only
the timing is reduced.  Checked on the CPU, including a two-rank gloo run."""
import os
import socket

import pytest

import bench


def _sizes():
    import math
    from paper_1601_02708_gb300.inputs import SplitMix64
    rng = SplitMix64(3)
    out = []
    for _ in range(256):
        side = int(round(math.exp(math.log(64) + (math.log(1024) - math.log(64)) * rng.uniform())))
        rng.uniform()
        rng.uniform()
        out.append(side * side)
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_partition_and_balance(world):
    sizes = _sizes()
    shards = [bench.shard_instances(sizes, r, world) for r in range(world)]
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in sh) for sh in shards]
    # greedy largest-first: the spread is at most the largest instance
    assert max(loads) - min(loads) <= max(sizes)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = _sizes()
        mine = bench.shard_instances(sizes, rank, world)
        # a stand-in for each rank's measured time: its share of the work
        t = float(sum(sizes[i] for i in mine))
        tmax = bench.reduce_max(t, dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, t, tmax, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    times = [r[1] for r in res]
    for _, _, tmax, gathered in res:
        assert tmax == max(times)
        assert sorted(i for sh in gathered for i in sh) == list(range(256))
        assert not set(gathered[0]) & set(gathered[1])
