"""Host logic of batched evaluation on several GPUs: the split of the
systems between ranks and the max-over-ranks timing, the latter run as two
gloo ranks on the CPU (no GPU involved)."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2412_04595_gb300.sharding import shard_systems, system_cost  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_partition_the_systems_and_balance_the_cost(world):
    rng = np.random.default_rng(7)
    sizes = [int(v) for v in np.exp(rng.uniform(np.log(500), np.log(50000), 256))]
    shards = shard_systems(sizes, world)
    assert len(shards) == world
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(sizes)))
    assert all(s == sorted(s) for s in shards)
    loads = [sum(system_cost(sizes[i]) for i in s) for s in shards]
    total, biggest = sum(loads), max(system_cost(n) for n in sizes)
    # longest-processing-time rule: no rank exceeds the mean by more than one system
    assert max(loads) <= total / world + biggest + 1e-6


def test_one_rank_takes_everything_in_order():
    assert shard_systems([5, 9, 2], 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        shard_systems([1], 0)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    import bench
    sizes = [1000 + 37 * i for i in range(20)]
    mine = shard_systems(sizes, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = bench.max_over_ranks(10.0 + rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, "rank%d.json" % rank), "w") as f:
        json.dump({"shards": gathered, "t": t}, f)


def test_two_gloo_ranks_agree_on_shards_and_max_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    g0, t0 = res[0]["shards"], res[0]["t"]
    g1, t1 = res[1]["shards"], res[1]["t"]
    assert g0 == g1 and sorted(g0[0] + g0[1]) == list(range(20)) and not set(g0[0]) & set(g0[1])
    assert t0 == t1 == 11.0
