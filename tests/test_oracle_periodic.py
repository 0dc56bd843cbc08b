"""Pins of the oracle's periodic sides (arXiv:1701.04329: Sec. 2 lists
periodic conditions; Sec. 2.2 imposes them through the coarse grid's
connectivity, the box beyond the last one being the first).  No GPU."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree
from tests.test_oracle_neumann import boundary_data
from tests.treecheck import check_tree

TYPES = {2: [[2, 2, 0, 0], [2, 2, 1, 0]], 3: [[2, 2, 0, 0, 2, 2], [0, 1, 2, 2, 0, 0]]}


def periodic_axes(types):
    return tuple(a for a in range(len(types) // 2) if types[2 * a] == 2)


def random_periodic(D, N, uniform, extra, seed, types, frac=0.3, n_buf=1, deref_rounds=0):
    """Periodic sides are set on the root box, then the tree is refined and
    adapted at random places (Sec. 2.3 rules)."""
    rng = np.random.default_rng(seed)
    t = OracleTree(D, N, uniform + extra)
    t.set_boundary_types(types)
    t.refine_uniform(uniform)
    for _ in range(extra):
        t.adapt(np.repeat((rng.random(t.nleaf) < frac).astype(np.int8), N ** D), n_buf)
    for _ in range(deref_rounds):
        t.adapt(-np.repeat((rng.random(t.nleaf) < 0.7).astype(np.int8), N ** D), n_buf)
    return t


@pytest.mark.parametrize("D,seed", [(2, 101), (2, 102), (3, 103)])
def test_periodic_tree_invariants(D, seed):
    """Neighbours wrap around on periodic axes (the root box is its own
    neighbour there), stay reciprocal, and 2:1 balance holds across the
    wrapped sides too -- also after derefinement."""
    for types in TYPES[D]:
        t = random_periodic(D, 4, 2, 3 if D == 2 else 2, seed, types, deref_rounds=2)
        check_tree(t.export(), D, periodic=periodic_axes(types))
    t = OracleTree(D, 4, 3)
    t.set_boundary_types(TYPES[D][0])
    e = t.export()
    assert e["neighbours"][0].max() == 0  # the root box wraps onto itself


def flag_box(t, level, idx):
    """Refinement flags (+1) on the cells of the leaf at (level, idx)."""
    e = t.export()
    nc = t.N ** t.D
    f = np.zeros(t.n_leaf_cells, np.int8)
    leaves = [b for b in range(len(e["level"])) if e["children"][b, 0] < 0]
    for li, b in enumerate(leaves):
        if e["level"][b] == level and tuple(int(v) for v in e["idx"][b][:t.D]) == idx:
            f[li * nc:(li + 1) * nc] = 1
    assert f.any()
    return f


def test_periodic_refinement_crosses_the_wrapped_side():
    """Refining next to x = 1 forces the 2:1 refinement of the box across the
    wrapped side at x = 0."""
    t = OracleTree(2, 4, 5)
    t.set_boundary_types([2, 2, 0, 0])
    t.refine_uniform(3)                 # 4 x 4 boxes on level 3
    t.adapt(flag_box(t, 3, (4, 2)), 0)  # level-4 boxes x = 7..8, y = 3..4
    t.adapt(flag_box(t, 4, (8, 3)), 0)  # level-5 boxes at the +x edge
    e = t.export()
    check_tree(e, 2, periodic=(0,))
    lv = {(int(l),) + tuple(int(v) for v in ix[:2]) for l, ix in zip(e["level"], e["idx"])}
    assert (5, 16, 5) in lv
    assert (4, 1, 3) in lv  # refined because of its neighbour across x = 1 -> 0


@pytest.mark.parametrize("D,seed", [(2, 111), (3, 112)])
def test_periodic_box_operator_equals_geometric_assembly(D, seed):
    """Box machinery = geometric assembly with wrapped lookups = explicit rows."""
    for types in TYPES[D]:
        t = random_periodic(D, 4, 2, 2, seed, types)
        e = t.export()
        K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types)
        assert B.shape[1] == t.n_bfaces
        rng = np.random.default_rng(seed)
        u = rng.normal(size=t.n_leaf_cells)
        b = rng.normal(size=t.n_bfaces)
        t.set_dirichlet(b)
        Au = t.apply_A(u)
        ref = K @ u + B @ b
        assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()
        assert abs(t.leaf_rows() - K).max() <= 1e-12 * abs(K).max()


@pytest.mark.parametrize("D,seed", [(2, 113), (3, 114)])
def test_periodic_flux_cancels(D, seed):
    """Conservation: what leaves through one periodic side enters through the
    other, so only the non-periodic faces carry flux:
    sum h^D (A u)_i = sum over Dirichlet faces h^(D-2) (2 b - 2 u_i(f))."""
    types = TYPES[D][0]
    t = random_periodic(D, 4, 2, 2, seed, types)
    e = t.export()
    rng = np.random.default_rng(seed)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    vol = composite.cell_volumes(D, 4, e["level"], e["children"])
    _, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types)
    area = composite.face_areas(D, 4, e["level"], e["idx"], e["children"], types)
    h_f = area ** (1.0 / (D - 1))
    cell_of_face = np.asarray(abs(B).tocsc().argmax(axis=0)).ravel()
    flux = h_f ** (D - 2) * (2 * b - 2 * u[cell_of_face])
    assert abs(np.sum(vol * Au) - np.sum(flux)) <= 1e-12 * np.sum(np.abs(vol * Au))


@pytest.mark.parametrize("D,seed", [(2, 115), (3, 116)])
def test_periodic_multigrid_converges_to_dense_solution(D, seed):
    for types in TYPES[D]:
        t = random_periodic(D, 4, 2 if D == 2 else 1, 2, seed, types, frac=0.4)
        e = t.export()
        K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types)
        rng = np.random.default_rng(seed)
        rho = rng.normal(size=t.n_leaf_cells)
        b = rng.normal(size=t.n_bfaces)
        ref = spla.spsolve(K.tocsc(), rho - B @ b)
        t.set_rhs(rho)
        t.set_dirichlet(b)
        t.zero_solution()
        t.solve(1e-13, 80)
        assert np.abs(t.get_solution() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_periodic_second_order_discretisation_error():
    """u = sin(2 pi x) (y^2 + 1) + y, periodic in x, Dirichlet in y: the max
    error drops by about 4 per halving of h."""
    u = lambda x: np.sin(2 * np.pi * x[..., 0]) * (x[..., 1] ** 2 + 1) + x[..., 1]
    lap = lambda x: np.sin(2 * np.pi * x[..., 0]) * (2 - 4 * np.pi ** 2 * (x[..., 1] ** 2 + 1))
    types = [2, 2, 0, 0]
    errs = []
    for lvl in (3, 4, 5):
        t = OracleTree(2, 8, lvl)
        t.set_boundary_types(types)
        t.refine_uniform(lvl)
        xc = t.cell_centers()
        t.set_rhs(lap(xc))
        t.set_dirichlet(boundary_data(t, types, u, lambda x: None))
        t.zero_solution()
        t.solve(1e-12, 60)
        errs.append(np.abs(t.get_solution() - u(xc)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders


def test_periodic_types_refused_when_invalid():
    t = OracleTree(2, 4, 3)
    for bad in ([2, 0, 0, 0], [2, 1, 0, 0], [0, 0, 1, 2]):
        with pytest.raises(ValueError):
            t.set_boundary_types(bad)
    t.refine_uniform(2)
    with pytest.raises(ValueError):  # connectivity changes only on the root box alone
        t.set_boundary_types([2, 2, 0, 0])
    t.set_boundary_types([1, 0, 0, 1])  # Dirichlet/Neumann changes stay allowed
