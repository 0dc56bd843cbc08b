"""The library's tree builder (host C++) against the oracle's, bit for bit:
box order, levels, spatial indices, parent/children/neighbour ids, cell and
face centres (arXiv:1701.04329 Sec. 2.1-2.3).  No GPU."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.treecheck import check_tree


def same_tree(a, b):
    ea, eb = a.export(), b.export()
    for k in ("level", "idx", "parent", "children", "neighbours"):
        assert np.array_equal(ea[k], eb[k]), k
    assert np.array_equal(a.cell_centers(), b.cell_centers())
    assert np.array_equal(a.face_centers(), b.face_centers())
    assert np.array_equal(a.leaf_levels(), b.leaf_levels())
    return ea


@pytest.mark.parametrize("D,N,seed", [(2, 4, 1), (2, 8, 2), (2, 16, 3), (3, 4, 4), (3, 8, 5)])
def test_random_adapt_sequences(D, N, seed):
    rng = np.random.default_rng(seed)
    maxl = 6 if D == 2 else 4
    a, b = OracleTree(D, N, maxl), afgpu.Tree(D, N, maxl)
    for t in (a, b):
        t.refine_uniform(2)
    for step in range(6):
        n = a.n_leaf_cells
        assert n == b.n_leaf_cells
        lv = np.repeat(a.leaf_levels(), N ** D)
        flags = rng.choice(np.array([-1, 0, 1], np.int8), size=n, p=[0.5, 0.45, 0.05])
        # whole boxes flagged -1 now and then, so derefinement happens too
        boxes = rng.random(n // N ** D) < 0.5
        flags[np.repeat(boxes, N ** D)] = -1
        nbuf = int(rng.integers(0, 3))
        ra = a.adapt(flags, nbuf)
        rb = b.adapt(flags, nbuf)
        assert ra == rb
        e = same_tree(a, b)
        check_tree(e, D)


@pytest.mark.parametrize("make", [W.gauss2d, lambda: W.twosrc3d(uniform_level=4, extra_levels=2, s=0.04),
                                  lambda: W.forest2d_problem(W.forest2d_params(3)[2]),
                                  lambda: W.blobs3d(uniform_level=3)])
def test_workload_trees(make):
    p = make()
    a, b = OracleTree(p.dim, p.box_n, p.max_level), afgpu.Tree(p.dim, p.box_n, p.max_level)
    p.build(a)
    p.build(b)
    same_tree(a, b)


@pytest.mark.parametrize("D,N,seed,types", [(2, 4, 11, [2, 2, 0, 0]), (2, 8, 12, [0, 1, 2, 2]),
                                            (3, 4, 13, [2, 2, 0, 0, 2, 2]), (3, 8, 14, [2, 2, 2, 2, 0, 1])])
def test_periodic_adapt_sequences(D, N, seed, types):
    """Periodic sides (Sec. 2.2: wrapped connectivity): both builders agree
    bit for bit, including 2:1 refinement across the wrapped sides."""
    rng = np.random.default_rng(seed)
    maxl = 6 if D == 2 else 4
    a, b = OracleTree(D, N, maxl), afgpu.Tree(D, N, maxl)
    for t in (a, b):
        t.set_boundary_types(types)
        t.refine_uniform(2)
    periodic = tuple(x for x in range(D) if types[2 * x] == 2)
    for step in range(5):
        n = a.n_leaf_cells
        assert n == b.n_leaf_cells
        flags = rng.choice(np.array([-1, 0, 1], np.int8), size=n, p=[0.4, 0.5, 0.1])
        flags[np.repeat(rng.random(n // N ** D) < 0.4, N ** D)] = -1
        nbuf = int(rng.integers(0, 3))
        assert a.adapt(flags, nbuf) == b.adapt(flags, nbuf)
        check_tree(same_tree(a, b), D, periodic=periodic)
    assert len(a.face_centers()) == b.n_bfaces


@pytest.mark.parametrize("D,N,roots,types,seed", [(2, 4, (2, 1), None, 41), (2, 8, (3, 2), [2, 2, 0, 1], 42),
                                                  (2, 4, (1, 3), [0, 0, 2, 2], 43), (3, 4, (2, 1, 1), None, 44),
                                                  (3, 4, (1, 2, 2), [0, 1, 2, 2, 0, 0], 45)])
def test_multiroot_adapt_sequences(D, N, roots, types, seed):
    """Level 1 a block of root boxes (Sec. 2.2): both builders agree bit for
    bit (root order, neighbours across root boundaries, 2:1 refinement across
    them and across wrapped sides), as do cell and face centres."""
    rng = np.random.default_rng(seed)
    maxl = 5 if D == 2 else 4
    a, b = OracleTree(D, N, maxl, roots=roots), afgpu.Tree(D, N, maxl, roots=roots)
    for t in (a, b):
        if types is not None:
            t.set_boundary_types(types)
        t.refine_uniform(2)
    periodic = tuple(x for x in range(D) if types is not None and types[2 * x] == 2)
    check_tree(same_tree(a, b), D, roots=roots, periodic=periodic)
    for step in range(5):
        n = a.n_leaf_cells
        assert n == b.n_leaf_cells
        flags = rng.choice(np.array([-1, 0, 1], np.int8), size=n, p=[0.4, 0.5, 0.1])
        flags[np.repeat(rng.random(n // N ** D) < 0.4, N ** D)] = -1
        nbuf = int(rng.integers(0, 3))
        assert a.adapt(flags, nbuf) == b.adapt(flags, nbuf)
        check_tree(same_tree(a, b), D, roots=roots, periodic=periodic)
    assert len(a.face_centers()) == b.n_bfaces


def test_manufactured_twin_shares_the_workload_tree():
    """The bench solves the manufactured twin on the workload's tree: both
    problems refine by the same flags (positions and width of the two
    sources), so the library builds the same tree for either."""
    for lvl in (3, 4):
        a, b = W.twosrc3d(uniform_level=lvl), W.twin3d(uniform_level=lvl)
        ta, tb = afgpu.Tree(3, 8, a.max_level), afgpu.Tree(3, 8, b.max_level)
        a.build(ta)
        b.build(tb)
        ea, eb = ta.export(), tb.export()
        assert all(np.array_equal(ea[k], eb[k]) for k in ("level", "idx", "parent", "children", "neighbours"))
