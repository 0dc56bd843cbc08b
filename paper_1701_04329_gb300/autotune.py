"""Autotuner for batched forest solves (an addition to the paper's method).

For a workload of independent 2D quadtrees it builds the forest with boxes
of 8^2 and of 16^2 cells (one level fewer with 16^2, so the finest spacing
is the same) and hands both to the library's tuner (``afg_autotune``), which
times the solve to the tolerance for every pair of smoothing steps (N_down,
N_up) and every threads-per-box choice of the FP32 half-sweep (one thread
per 16-byte vector of a box's colour half, or half as many) and picks the
configuration with the most unknowns per second (time to the tolerance per
unknown: the two box sizes refine to different meshes at the same finest
spacing).

``python -m paper_1701_04329_gb300.autotune 512`` on a GPU writes the choice
to ``tuned_forest.json`` beside this file; ``bench.py`` times the batched
workload at that configuration.
"""
import ctypes
import json
import os

import numpy as np

from . import afgpu
from . import workloads as W

TUNED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_forest.json")


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


def autotune_forest(n_trees=512, seed0=1000, tol=1e-8, precision=afgpu.AFG_MIXED, box_sizes=(8, 16),
                    sweeps=((1, 1), (2, 2), (3, 3)), vectors_per_thread=(1, 2), reps=3, max_level_cap=None):
    """Returns (best, table) from afg_autotune."""
    import torch
    forests, keep = [], []
    for box_n in box_sizes:
        trees, rho, b = build_forest(n_trees, box_n, seed0, max_level_cap)
        f = afgpu.Forest(trees)
        f.set_rhs(torch.tensor(rho, device="cuda"))
        f.set_dirichlet(torch.tensor(b, device="cuda"))
        forests.append(f)
        keep.append(trees)
    base = afgpu.default_opts(rel_tol=tol, precision=precision, max_cycles=60)
    spec = json.dumps({"sweeps": [list(s) for s in sweeps], "vectors_per_thread": list(vectors_per_thread),
                       "reps": reps}).encode()
    out = ctypes.create_string_buffer(1 << 16)
    arr = (ctypes.c_void_p * len(forests))(*[f._h.value for f in forests])
    for f in forests:
        f._sync_stream()
    afgpu._check(afgpu.lib().afg_autotune(arr, len(forests), ctypes.byref(base), spec, out, len(out)))
    rep = json.loads(out.value.decode())
    for f in forests:
        f.close()
    for trees in keep:
        for t in trees:
            t.close()
    return rep["best"], rep["table"]


def record(best, table, n_trees, tol, path=TUNED):
    with open(path, "w") as f:
        json.dump({"workload": "batched 2D forest, %d trees, seeds 1000+t" % n_trees, "tol": tol,
                   "objective": "unknowns_per_s", "best": best, "table": table}, f, indent=1)
        f.write("\n")


def tuned_choice(path=TUNED):
    """The recorded choice (box_n, n_down, n_up, threads_per_box), or None."""
    try:
        with open(path) as f:
            b = json.load(f)["best"]
        return int(b["box_n"]), int(b["n_down"]), int(b["n_up"]), int(b.get("threads_per_box", 0))
    except (OSError, KeyError, ValueError):
        return None


if __name__ == "__main__":
    import sys
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    tol = 1e-8
    best, table = autotune_forest(n, tol=tol)
    if n == 512:
        record(best, table, n, tol)
    print(json.dumps({"best": best, "table": table}, indent=1))
