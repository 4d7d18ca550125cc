"""The multi-rank host logic of bench.py on the CPU with the gloo backend
(world size 2, 127.0.0.1): the batch is sharded without overlap or gap
(instance i to rank i mod N), and the slowest rank's time and the ranks'
summed work are what every rank reports.  The solve itself does not shard
(one problem per GPU, replicas only), so these reductions are the only
exchanges between ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    import json

    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        items = list(range(64))
        mine = bench.shard(items, rank, ws)
        times = [0.5 + rank, 2.0 - rank]             # rank 1 is slower on the first, faster on the second
        tmax = bench.reduce_ranks(times, dist, ws, "max", device="cpu")
        total = bench.reduce_ranks([len(mine), sum(mine)], dist, ws, "sum", device="cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"mine": mine, "tmax": tmax, "total": total}, fh)
    finally:
        dist.destroy_process_group()


def test_sharding_and_reductions_over_two_gloo_ranks(tmp_path):
    import json

    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    mp.spawn(_rank, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    shards = [set(r["mine"]) for r in res]
    assert shards[0].isdisjoint(shards[1]) and shards[0] | shards[1] == set(range(64))
    assert res[0]["mine"] == list(range(0, 64, 2)) and res[1]["mine"] == list(range(1, 64, 2))
    for r in res:
        assert r["tmax"] == [1.5, 2.0]
        assert r["total"] == [64.0, float(sum(range(64)))]


def test_single_rank_is_the_identity():
    import bench
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
    assert bench.reduce_ranks([1.0, 2.5], None, 1, "max") == [1.0, 2.5]
