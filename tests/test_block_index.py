"""Index arithmetic of the block bottom solve (csrc/block_bottom.cuh, built
for the host): where each cell and each boundary face cell of a block of
root boxes lives in the library's per-box storage.  Checked bit for bit
against the library's own tree (root boxes in canonical order, cell and
face centres) and an enumeration of the red-black box layout.  No GPU."""
import os
import subprocess

import numpy as np
import pytest

from paper_1701_04329_gb300 import afgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("blkidx")
    out = str(d / "block_index_host")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", out, os.path.join(ROOT, "tests", "block_index_host.cpp")],
                   check=True)
    return out


def rb_layout(D, M):
    """storage position of each 0-based cell (i, j, k) of a box: the red half
    ((i + j + k + D) even) then the black half, each in (k, j, i >> 1) order"""
    pos, n = {}, 0
    for colour in (0, 1):
        for k in range(M if D == 3 else 1):
            for j in range(M):
                for h in range(M // 2):
                    i = 2 * h + ((colour + j + k + D) & 1)
                    pos[(i, j, k)] = n
                    n += 1
    return pos


@pytest.mark.parametrize("D,N,roots", [(2, 8, (3, 2)), (2, 4, (1, 3)), (3, 8, (2, 1, 2)), (3, 4, (1, 2, 2))])
def test_cells_and_faces_find_their_boxes(exe, D, N, roots):
    t = afgpu.Tree(D, N, 1, roots=roots)
    e = t.export()
    # canonical position of root (ri, rj, rk)
    slot = {tuple(int(v) - 1 for v in e["idx"][b]): b for b in range(len(e["level"]))}
    nr = list(roots) + [1] * (3 - D)
    lines = subprocess.run([exe, str(D), str(N)] + [str(r) for r in nr], capture_output=True, text=True,
                           check=True).stdout.split("\n")
    cells = [tuple(map(int, l.split()[1:])) for l in lines if l.startswith("c ")]
    faces = [tuple(map(int, l.split()[1:])) for l in lines if l.startswith("f ")]
    layout = rb_layout(D, N)
    n = [r * N for r in roots]
    # every block cell, rectangle order (x fastest)
    for c, (root, q) in enumerate(cells):
        g = [c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1]) if D == 3 else 0]
        r = [g[a] // N for a in range(D)] + [0] * (3 - D)
        assert root == r[0] + nr[0] * (r[1] + nr[1] * r[2])
        loc = tuple(g[a] % N for a in range(D)) + ((0,) if D == 2 else ())
        assert q == layout[loc]
    assert len(cells) == int(np.prod(n))
    # the box a root index names has that root's spatial index
    for root in range(int(np.prod(roots))):
        r = (root % nr[0], (root // nr[0]) % nr[1], root // (nr[0] * nr[1]))
        assert tuple(int(v) - 1 for v in e["idx"][slot[r[:D]]]) == r[:D]
    # every boundary face cell: compare with the canonical face order of the library
    fc = t.face_centers()
    h = 1.0 / N
    canon = {}
    per = N ** (D - 1)
    o = 0
    for b in range(len(e["level"])):         # all boxes are leaves (level 1 only)
        for s in range(2 * D):
            if e["neighbours"][b][[3, 4, 1, 6][s] if D == 2 else [12, 13, 10, 15, 4, 21][s]] != -2:
                continue
            for f in range(per):
                canon[o + f] = (b, s, f)
            o += per
    assert o == t.n_bfaces
    seen = 0
    for s in range(2 * D):
        a, hi = s // 2, s % 2
        t1 = 1 if a == 0 else 0
        t2 = (1 if a == 2 else 2) if D == 3 else None
        mine = [(root, lf) for (ss, root, lf) in faces if ss == s]
        on = np.nonzero(fc[:, a] == (roots[a] if hi else 0.0))[0]
        for fi in on:
            f = int(np.floor(fc[fi, t1] / h))
            if t2 is not None:
                f += n[t1] * int(np.floor(fc[fi, t2] / h))
            b, s_c, lf_c = canon[fi]
            root, lf = mine[f]
            r = (root % nr[0], (root // nr[0]) % nr[1], root // (nr[0] * nr[1]))
            assert s_c == s and slot[r[:D]] == b and lf == lf_c
            seen += 1
    assert seen == t.n_bfaces
