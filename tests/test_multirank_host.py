"""The multi-rank host logic of bench.py on CPU with the gloo backend,
world size 2: ranks run independent work (replicas, or shards of the
batched form) and only the timing is reduced; value = all ranks' units /
the slowest rank's time."""

import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [100.0, 300.0][rank]
    secs = [2.0, 3.0][rank]
    res = {"max": bench.reduce_max(1.5 + rank), "sum": bench.reduce_sum(rank + 1.0),
           "value": bench.weak_value(units, secs)}
    # each rank takes its shard of the same systems
    costs = [5000, 300, 2000, 2000, 800, 7000, 100]
    res["shard"] = bench.shard_by_cost(costs, world)[rank]
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, "r%d.json" % rank), "w") as f:
        json.dump(res, f)


def test_two_rank_reductions_and_shards(tmp_path):
    tmp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("r%d.json" % k))) for k in range(2)]
    for k in range(2):
        assert r[k]["max"] == 2.5
        assert r[k]["sum"] == 3.0
        assert r[k]["value"] == pytest.approx(400.0 / 3.0)
    shards = r[0]["shard"] + r[1]["shard"]
    assert sorted(shards) == list(range(7)) and not set(r[0]["shard"]) & set(r[1]["shard"])


def test_shard_by_cost_balances():
    costs = [5000, 300, 2000, 2000, 800, 7000, 100]
    parts = bench.shard_by_cost(costs, 3)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert sorted(i for p in parts for i in p) == list(range(7))
    assert max(loads) == 7000  # the largest system alone bounds the makespan
    assert bench.shard_by_cost(costs, 1) == [list(range(7))]


def test_single_process_reductions_are_identity():
    assert bench.reduce_max(3.25) == 3.25
    assert bench.weak_value(10.0, 2.0) == 5.0
