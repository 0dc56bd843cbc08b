"""The batched forest split across ranks (no GPU): LPT partition of whole
trees by box count, built identically on every rank from the host trees,
and the one gather of per-tree results on rank 0 with two gloo ranks."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_1701_04329_gb300 import shard
from tests.test_bench_ranks import ROOT, free_port


def test_lpt_partition_covers_balances_and_is_deterministic():
    rng = np.random.default_rng(4)
    costs = list(rng.integers(1, 1000, size=97))
    for world in (1, 2, 3, 8):
        bins = shard.lpt_partition(costs, world)
        assert sorted(i for b in bins for i in b) == list(range(len(costs)))
        loads = [sum(costs[i] for i in b) for b in bins]
        # Graham's bound for LPT: makespan <= (4/3 - 1/(3m)) OPT, and OPT >= max(mean, max item)
        opt_lb = max(sum(costs) / world, max(costs))
        assert max(loads) <= (4 / 3 - 1 / (3 * world)) * opt_lb + 1e-9
        assert bins == shard.lpt_partition(costs, world)
    assert shard.lpt_partition([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert shard.lpt_partition([1, 9, 3], 2) == [[1], [0, 2]]


def test_gather_on_one_rank_orders_by_tree():
    out = shard.gather_stats(None, 0, 1, [(2, "c"), (0, "a"), (1, "b")], 3)
    assert out == ["a", "b", "c"]


WORKER = r"""
import os, sys, json
sys.path.insert(0, %r)
import bench
from paper_1701_04329_gb300 import shard, workloads as W, afgpu
dist, rank, world, local = bench.dist_init()
# every rank builds the same host trees (no GPU), so every rank computes the same partition
params = W.forest2d_params(12, 1000)
boxes = []
for prm in params:
    prm = dict(prm, max_level=min(prm["max_level"], 6))
    p = W.forest2d_problem(prm, 8)
    t = afgpu.Tree(2, 8, p.max_level)
    p.build(t)
    boxes.append(t.info().n_boxes)
bins = shard.lpt_partition(boxes, world)
mine = [(i, {"tree": i, "rank": rank, "boxes": boxes[i]}) for i in bins[rank]]
out = shard.gather_stats(dist, rank, world, mine, len(boxes))
print(json.dumps({"rank": rank, "bins": bins, "boxes": boxes, "out": out}))
dist.destroy_process_group()
"""


def test_shard_partition_and_gather_with_two_gloo_ranks():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER % ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = {}
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        d = json.loads(out.strip().splitlines()[-1])
        outs[d["rank"]] = d
    assert outs[0]["bins"] == outs[1]["bins"] and outs[0]["boxes"] == outs[1]["boxes"]
    bins, boxes = outs[0]["bins"], outs[0]["boxes"]
    assert sorted(bins[0] + bins[1]) == list(range(12))
    assert outs[1]["out"] is None
    got = outs[0]["out"]
    assert [g["tree"] for g in got] == list(range(12))
    for g in got:
        assert g["boxes"] == boxes[g["tree"]] and g["tree"] in bins[g["rank"]]
    loads = [sum(boxes[i] for i in b) for b in bins]
    assert max(loads) <= (4 / 3 - 1 / 6) * max(sum(boxes) / 2, max(boxes)) + 1e-9
