"""Autotuner for batched forest solves (an addition to the paper's method).

For a workload of independent 2D quadtrees it builds the forest with boxes
of 8^2 and of 16^2 cells (one level fewer with 16^2, so the finest spacing
is the same), and for each box size times the solve to the tolerance with
every candidate pair of smoothing steps (N_down, N_up); the fastest
configuration wins.  Threads per box are not a free knob here: every kernel
assigns one thread per 16-byte vector of a box's colour half (or per cell
pair for small boxes), so the box size fixes them; the tuner reports them.
Timing: CUDA events around whole solves, after one warm-up solve.
"""
import json

import numpy as np

from . import afgpu
from . import workloads as W


def build_forest(n_trees, box_n, seed0=1000, max_level_cap=None):
    trees, rhos, bs = [], [], []
    for prm in W.forest2d_params(n_trees, seed0):
        if max_level_cap is not None:
            prm = dict(prm, max_level=min(prm["max_level"], max_level_cap))
        p = W.forest2d_problem(prm, box_n)
        t = afgpu.Tree(2, box_n, p.max_level)
        p.build(t)
        rho, b = p.data(t)
        trees.append(t)
        rhos.append(rho)
        bs.append(b)
    return trees, np.concatenate(rhos), np.concatenate(bs)


def threads_per_box(dim, box_n, fp32=True):
    half = box_n ** dim // 2
    vec = 4 if fp32 else 2
    return min(max(half // vec, 1), 256)


def time_forest(forest, rho, b, opts, reps=3):
    import torch
    f_rho = torch.tensor(rho, device="cuda")
    f_b = torch.tensor(b, device="cuda")
    forest.set_rhs(f_rho)
    forest.set_dirichlet(f_b)
    stats = forest.solve(opts, allow_not_converged=True)  # warm-up (builds the CUDA graphs)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        torch.cuda.synchronize()
        ev0.record()
        stats = forest.solve(opts, allow_not_converged=True)
        ev1.record()
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    worst = max(s["rel_residual"] for s in stats)
    return min(ms), worst, stats


def autotune_forest(n_trees=512, seed0=1000, tol=1e-8, precision=afgpu.AFG_MIXED, box_sizes=(8, 16),
                    sweeps=((1, 1), (2, 2), (3, 3)), reps=3, max_level_cap=None):
    """Returns (best, table): best is a dict of the chosen configuration."""
    table = []
    for box_n in box_sizes:
        trees, rho, b = build_forest(n_trees, box_n, seed0, max_level_cap)
        forest = afgpu.Forest(trees)
        cells = int(forest.cells.sum())
        for nd, nu in sweeps:
            opts = afgpu.default_opts(rel_tol=tol, precision=precision, n_down=nd, n_up=nu, max_cycles=60)
            ms, worst, stats = time_forest(forest, rho, b, opts, reps)
            table.append(dict(box_n=box_n, n_down=nd, n_up=nu, threads_per_box=threads_per_box(2, box_n),
                              ms=ms, unknowns=cells, unknowns_per_s=cells / (ms * 1e-3),
                              converged=bool(worst <= tol), worst_rel_residual=worst,
                              max_cycles=max(s["cycles"] for s in stats)))
        forest.close()
        for t in trees:
            t.close()
    ok = [r for r in table if r["converged"]] or table
    best = min(ok, key=lambda r: r["ms"])
    return best, table


if __name__ == "__main__":
    import sys
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    best, table = autotune_forest(n)
    print(json.dumps({"best": best, "table": table}, indent=1))
