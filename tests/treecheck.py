"""Brute-force checks of tree invariants, re-derived from spatial indices only
(arXiv:1701.04329 Sec. 1.3 and 2.1: children of (i,j) are (2i-1..2i, 2j-1..2j),
neighbours are at i+-1; proper nesting / 2:1 balance)."""
import itertools

import numpy as np


def morton(idx):
    k = 0
    for b in range(21):
        for a, v in enumerate(idx):
            k |= (((int(v) - 1) >> b) & 1) << (len(idx) * b + a)
    return k


def directions(D):
    out = []
    for off in itertools.product((-1, 0, 1), repeat=D):
        off = off[::-1]  # x fastest
        if any(off):
            out.append(off)
    return out


def check_tree(e, D, N=None, periodic=(), roots=None):
    """periodic: axes whose neighbours wrap around (Sec. 2.2); roots: root
    boxes per axis (default one)."""
    nr = list(roots) if roots is not None else [1] * D
    level, idx, parent, children, nbs = e["level"], e["idx"], e["parent"], e["children"], e["neighbours"]
    n = len(level)
    pos = {(int(level[b]),) + tuple(int(v) for v in idx[b]): b for b in range(n)}
    # canonical order: level ascending, Morton ascending within a level
    keys = [(int(level[b]), morton(idx[b])) for b in range(n)]
    assert keys == sorted(keys) and len(set(keys)) == n
    dirs = directions(D)
    for b in range(n):
        l = int(level[b])
        side = [nr[a] * 2 ** (l - 1) for a in range(D)]
        # parent / children from spatial indices
        if l == 1:
            assert parent[b] == -1
        else:
            assert parent[b] == pos[(l - 1,) + tuple((int(v) + 1) // 2 for v in idx[b])]
        kids = [pos.get((l + 1,) + tuple(2 * int(idx[b][a]) - 1 + ((c >> a) & 1) for a in range(D)), -1)
                for c in range(2 ** D)]
        assert list(children[b]) == kids
        assert all(k >= 0 for k in kids) or all(k < 0 for k in kids)  # never partially refined
        for d, off in enumerate(dirs):
            q = [int(idx[b][a]) + off[a] for a in range(D)]
            q = [(v - 1) % side[a] + 1 if a in periodic else v for a, v in enumerate(q)]
            if any(v < 1 or v > side[a] for a, v in enumerate(q)):
                assert nbs[b, d] == -2
            else:
                want = pos.get((l,) + tuple(q), -1)
                assert nbs[b, d] == want
                if want >= 0:  # reciprocity
                    back = dirs.index(tuple(-o for o in off))
                    assert nbs[want, back] == b
    # 2:1 balance between all touching leaves (faces, edges and corners)
    leaves = [b for b in range(n) if children[b, 0] < 0]
    lo = np.array([(idx[b] - 1) / 2.0 ** (level[b] - 1) for b in leaves])
    hi = lo + np.array([1.0 / 2.0 ** (level[b] - 1) for b in leaves])[:, None]
    lv = level[leaves]
    shifts = [s for s in itertools.product((-1, 0, 1), repeat=D) if all(s[a] == 0 or a in periodic for a in range(D))]
    for i in range(len(leaves)):
        for sh in shifts:  # periodic images touch across the wrapped sides
            shift = np.array(sh) * np.array(nr)
            lo_i, hi_i = lo[i] + shift, hi[i] + shift
            touch = np.all((lo <= hi_i + 1e-12) & (hi >= lo_i - 1e-12), axis=1)
            assert np.all(np.abs(lv[touch] - lv[i]) <= 1), "2:1 balance violated"
    # leaves tile the domain
    assert abs(sum(1.0 / 2.0 ** (D * (level[b] - 1)) for b in leaves) - float(np.prod(nr))) < 1e-12
