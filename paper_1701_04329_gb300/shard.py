"""Batched forests split across GPUs (one process per GPU).

The trees of a batched workload are independent problems, so they shard with
no exchange on the solve path: every rank builds the host trees of the whole
batch (a deterministic host-side computation, identical on every rank),
assigns whole trees to ranks by LPT on their box counts (Graham's longest-
processing-time rule: trees in decreasing box count, each to the rank with
the fewest boxes so far, ties to the lower rank), builds a forest of its own
trees on its GPU and solves it.  Only the per-tree results come back: rank 0
gathers the statistics once, after the solves, in the batch's tree order.
"""
import heapq


def lpt_partition(costs, world):
    """Whole items to `world` bins, largest first, each to the least-loaded
    bin (ties: lower bin index, then lower item index).  Returns a list of
    item-index lists, each in increasing order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    bins = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        bins[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(b) for b in bins]


def gather_stats(dist, rank, world, mine, n_items):
    """Per-item results of every rank, in item order, on rank 0 (None on the
    others).  `mine` is a list of (item index, result) of this rank.  One
    gather, after the solves."""
    if dist is None or world == 1:
        out = [None] * n_items
        for i, r in mine:
            out[i] = r
        return out
    parts = [None] * world if rank == 0 else None
    dist.gather_object(mine, parts, dst=0)
    if rank != 0:
        return None
    out = [None] * n_items
    for part in parts:
        for i, r in part:
            out[i] = r
    return out


def build_batch(n_trees, box_n, seed0=1000):
    """The host trees and data of the batched 2D workload (every rank builds
    all of them; no GPU is involved)."""
    from . import afgpu
    from . import workloads as W
    trees, rhos, bs = [], [], []
    for prm in W.forest2d_params(n_trees, seed0):
        p = W.forest2d_problem(prm, box_n)
        t = afgpu.Tree(2, box_n, p.max_level)
        p.build(t)
        rho, b = p.data(t)
        trees.append(t)
        rhos.append(rho)
        bs.append(b)
    return trees, rhos, bs


def solve_shard(trees, rhos, bs, mine, opts, dev):
    """Forest of this rank's trees on its GPU: set the data, solve; returns
    [(tree index, stats dict)] and the forest (for timing)."""
    import numpy as np
    import torch
    from . import afgpu
    f = afgpu.Forest([trees[i] for i in mine])
    f.set_rhs(torch.tensor(np.concatenate([rhos[i] for i in mine]), device=dev))
    f.set_dirichlet(torch.tensor(np.concatenate([bs[i] for i in mine]), device=dev))
    st = f.solve(opts)
    return [(i, s) for i, s in zip(mine, st)], f
