"""Pins of the oracle's domains made of several root boxes (arXiv:1701.04329
Sec. 2.2: the coarsest level is a block of root boxes; Sec. 3.2: below it
the coarse grids hold one box per root, so a non-square domain has several
2^D-cell boxes on the coarsest grid, relaxed together).  No GPU.

Pins: tree invariants re-derived from spatial indices on rectangular root
blocks; the box machinery equals the geometric assembly of the composite
system; multigrid converges to the dense solution of that system; a
2 x 1 block, periodic in x, with a source of period 1 in x reproduces the
single-root periodic solution on both halves (translation symmetry of the
discrete problem); one root box reproduces the single-root tree bit for bit."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree
from tests.treecheck import check_tree

ROOTS = {2: [(2, 1), (3, 2), (1, 3)], 3: [(2, 1, 1), (1, 2, 2)]}
TYPES = {2: [None, [2, 2, 0, 0], [0, 1, 0, 0]], 3: [None, [0, 0, 2, 2, 0, 1]]}


def periodic_axes(types):
    return tuple(a for a in range(len(types) // 2) if types[2 * a] == 2) if types else ()


def random_multiroot(D, N, roots, uniform, extra, seed, types=None, frac=0.3, n_buf=1, deref_rounds=0):
    rng = np.random.default_rng(seed)
    t = OracleTree(D, N, uniform + extra, roots=roots)
    if types is not None:
        t.set_boundary_types(types)
    t.refine_uniform(uniform)
    for _ in range(extra):
        t.adapt(np.repeat((rng.random(t.nleaf) < frac).astype(np.int8), N ** D), n_buf)
    for _ in range(deref_rounds):
        t.adapt(-np.repeat((rng.random(t.nleaf) < 0.7).astype(np.int8), N ** D), n_buf)
    return t


@pytest.mark.parametrize("D", [2, 3])
def test_multiroot_tree_invariants(D):
    for k, roots in enumerate(ROOTS[D]):
        for types in TYPES[D]:
            t = random_multiroot(D, 4, roots, 2, 3 if D == 2 else 2, 200 + 10 * D + k, types, deref_rounds=2)
            check_tree(t.export(), D, roots=roots, periodic=periodic_axes(types))
        # uniform levels: prod(roots) * 2^(D(l-1)) boxes, roots first, without parents
        u = OracleTree(D, 4, 3, roots=roots)
        u.refine_uniform(3)
        e = u.export()
        R = int(np.prod(roots))
        for l in (1, 2, 3):
            assert int(np.sum(e["level"] == l)) == R * 2 ** (D * (l - 1))
        assert np.all(e["parent"][:R] == -1)
        check_tree(e, D, roots=roots)


@pytest.mark.parametrize("D", [2, 3])
def test_multiroot_geometry(D):
    """Cell centres fill [0, rx] x [0, ry] (x [0, rz]); boundary faces lie on
    its sides; their number is that of a uniform block."""
    roots = ROOTS[D][0]
    t = OracleTree(D, 4, 3, roots=roots)
    t.refine_uniform(2)
    h = 1.0 / 8
    x = t.cell_centers()
    for a in range(D):
        assert x[:, a].min() == h / 2 and x[:, a].max() == roots[a] - h / 2
    # every cell centre once
    assert len({tuple(np.round(v / h - 0.5).astype(int)) for v in x}) == len(x)
    f = t.face_centers()
    on_side = np.zeros(len(f), bool)
    for a in range(D):
        on_side |= (f[:, a] == 0.0) | (f[:, a] == roots[a])
    assert on_side.all()
    cells = [r * 8 for r in roots]
    want = sum(2 * int(np.prod([cells[b] for b in range(D) if b != a])) for a in range(D))
    assert t.n_bfaces == want


@pytest.mark.parametrize("D,seed", [(2, 221), (3, 222)])
def test_multiroot_box_operator_equals_geometric_assembly(D, seed):
    for roots in ROOTS[D]:
        for types in TYPES[D]:
            t = random_multiroot(D, 4, roots, 2 if D == 2 else 1, 2, seed, types)
            e = t.export()
            K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types, roots=roots)
            assert B.shape[1] == t.n_bfaces
            rng = np.random.default_rng(seed)
            u = rng.normal(size=t.n_leaf_cells)
            b = rng.normal(size=t.n_bfaces)
            t.set_dirichlet(b)
            Au = t.apply_A(u)
            ref = K @ u + B @ b
            assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()
            assert abs(t.leaf_rows() - K).max() <= 1e-12 * abs(K).max()


def test_multiroot_coarse_grids():
    """Below the roots each level holds one box per root, connected like the
    roots; a level-1 box restricts into the level-0 box of its own root."""
    roots = (3, 2)
    t = OracleTree(2, 8, 3, roots=roots)
    t.refine_uniform(2)
    t.set_rhs(np.zeros(t.n_leaf_cells))
    mg = t.mg_boxes()
    R = 6
    assert t.lmin == -1                      # 8 -> boxes of 4 and 2 cells below the roots
    sub = [m for m in mg if m["tbox"] < 0]
    assert len(sub) == 2 * R
    e = t.export()
    for i, m in enumerate(sub):
        r = i % R
        assert m["level"] == t.lmin + i // R and m["M"] == 8 >> (1 - m["level"])
        assert m["parent"] == (i - R if i >= R else -1)
        for s in range(4):
            q = e["neighbours"][r][[3, 4, 1, 6][s]]    # -x, +x, -y, +y of the root
            if q >= 0:
                assert m["kind"][s] == 0 and m["nbid"][s] == (i // R) * R + q
            else:
                assert m["kind"][s] == 1 and m["nbid"][s] == -1
    for m in mg:
        if m["tbox"] >= 0 and m["level"] == 1:
            assert m["parent"] == R + m["tbox"]


@pytest.mark.parametrize("D,seed", [(2, 231), (3, 232)])
def test_multiroot_multigrid_converges_to_dense_solution(D, seed):
    for roots in ROOTS[D][:2]:
        for types in TYPES[D]:
            t = random_multiroot(D, 4, roots, 2 if D == 2 else 1, 2, seed, types, frac=0.4)
            e = t.export()
            K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types, roots=roots)
            rng = np.random.default_rng(seed)
            rho = rng.normal(size=t.n_leaf_cells)
            b = rng.normal(size=t.n_bfaces)
            ref = spla.spsolve(K.tocsc(), rho - B @ b)
            t.set_rhs(rho)
            t.set_dirichlet(b)
            t.zero_solution()
            t.solve(1e-13, 120)
            assert np.abs(t.get_solution() - ref).max() <= 1e-10 * np.abs(ref).max()


def _periodic_source(x):
    return np.sin(2 * np.pi * x[:, 0] + 0.3) * np.cos(3 * x[:, 1]) + np.exp(-30 * ((x[:, 0] % 1 - 0.4) ** 2
                                                                                 + (x[:, 1] - 0.6) ** 2))


@pytest.mark.parametrize("N", [4, 8])
def test_two_periodic_roots_tile_one_root(N):
    """Translation symmetry: on [0,2] x [0,1], periodic in x, a source and a
    refinement pattern of period 1 in x give the single-root solution on
    both halves (the discrete problem is the same cell for cell)."""
    trees = []
    for roots in ((1, 1), (2, 1)):
        t = OracleTree(2, N, 5, roots=roots)
        t.set_boundary_types([2, 2, 0, 0])
        t.refine_uniform(2)
        for _ in range(3):
            x = t.cell_centers()
            r = np.hypot(x[:, 0] % 1 - 0.4, x[:, 1] - 0.6)
            t.adapt((r < 0.15).astype(np.int8), 1)
        x = t.cell_centers()
        t.set_rhs(_periodic_source(x))
        fc = t.face_centers()
        t.set_dirichlet(np.cos(2 * np.pi * fc[:, 0]) * fc[:, 1])
        t.zero_solution()
        t.solve(1e-12, 60)
        trees.append((t, x))
    (a, xa), (b, xb) = trees
    assert b.n_leaf_cells == 2 * a.n_leaf_cells
    ua = {tuple(np.round(v * 4096).astype(int)): u for v, u in zip(xa, a.get_solution())}
    ub = b.get_solution()
    ref = np.array([ua[tuple(np.round(np.array([v[0] % 1, v[1]]) * 4096).astype(int))] for v in xb])
    assert np.abs(ub - ref).max() <= 1e-9 * np.abs(ref).max()


def test_one_root_is_the_single_root_tree():
    """roots=(1,1) and the default constructor give the same tree and the same
    solution, bit for bit."""
    out = []
    for roots in (None, (1, 1)):
        t = OracleTree(2, 8, 4, roots=roots)
        t.refine_uniform(2)
        t.adapt(np.repeat((np.arange(4) % 3 == 0).astype(np.int8), 64), 1)
        x = t.cell_centers()
        t.set_rhs(np.sin(5 * x[:, 0]) * x[:, 1])
        t.set_dirichlet(np.zeros(t.n_bfaces))
        t.zero_solution()
        t.solve(1e-10, 40)
        out.append((t.export(), t.get_solution()))
    for k in out[0][0]:
        assert np.array_equal(out[0][0][k], out[1][0][k])
    assert np.array_equal(out[0][1], out[1][1])


def test_multiroot_cycle_convergence():
    """V(2,2) cycles, N_base = 4: blocks of 2 x 1 and 3 x 1 roots (two or
    three 2 x 2 boxes on the coarsest grid, relaxed together) reduce the
    residual per cycle as fast as a single root box does on the same source
    (within 5 %; about 0.09-0.11 per cycle here, 0.07 in Sec. 4.1)."""
    worst = {}
    for roots in ((1, 1), (2, 1), (3, 1)):
        t = OracleTree(2, 8, 6, roots=roots)
        t.refine_uniform(4)
        x = t.cell_centers()
        t.set_rhs(np.exp(-((x[:, 0] - 0.7) ** 2 + (x[:, 1] - 0.4) ** 2) / 0.01))
        t.set_dirichlet(np.zeros(t.n_bfaces))
        t.zero_solution()
        hist = []
        t.solve(1e-12, 30, history=hist)
        f = [hist[i + 1] / hist[i] for i in range(len(hist) - 1)]
        worst[roots] = max(f[1:])
    assert worst[(1, 1)] <= 0.12
    for roots in ((2, 1), (3, 1)):
        assert worst[roots] <= 1.05 * worst[(1, 1)], worst
