"""Pins of the oracle's Neumann sides (arXiv:1701.04329, Sec. 2 and Sec. 3:
Dirichlet, Neumann and periodic conditions, or a mix, through ghost cells).
Reading: the Neumann datum b is the outward normal derivative at the face
centre and the ghost is g = u_1 + h b.  No GPU."""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree
from tests.test_oracle_pins import _cf_tree, _g, _set_all, random_amr

TYPES = {2: [1, 0, 0, 1], 3: [1, 0, 1, 0, 0, 1]}


def face_sides(t):
    """Side (2a + hi) of every boundary face, canonical face order."""
    xyz = t.face_centers()
    side = np.full(len(xyz), -1)
    for a in range(t.D):
        side[xyz[:, a] == 0.0] = 2 * a
        side[xyz[:, a] == 1.0] = 2 * a + 1
    assert (side >= 0).all()
    return xyz, side


def boundary_data(t, types, u, grad):
    """Dirichlet values u(x_f) or outward normal derivatives at the face centres."""
    xyz, side = face_sides(t)
    b = np.empty(len(xyz))
    for f, (x, s) in enumerate(zip(xyz, side)):
        b[f] = grad(x)[s // 2] * (1 if s % 2 else -1) if types[s] == 1 else u(x)
    return b


@pytest.mark.parametrize("D", [2, 3])
def test_neumann_ghost_exact_for_linear_fields(D):
    """g = u_1 + h b with b the outward derivative reproduces a linear field at
    the ghost centre, as the Dirichlet and refinement-boundary ghosts do."""
    N, types = 4, TYPES[D]
    t = _cf_tree(D, N)
    t.set_boundary_types(types)
    coef = np.array([0.3, -1.7, 0.9][:D])
    lin = lambda x: 0.25 + x @ coef
    t.set_dirichlet(boundary_data(t, types, lin, lambda x: coef))
    boxes = _set_all(t, lin)
    e = t.export()
    for lvl in (1, 2, 3):
        t.fill_ghosts(lvl, 0)
    n_neu = 0
    for b, m in enumerate(boxes):
        if m["tbox"] < 0:
            continue
        a = t.mg_get(b, 0, N)
        lo = (e["idx"][m["tbox"]] - 1) / 2.0 ** (m["level"] - 1)
        h = 1.0 / (N * 2.0 ** (m["level"] - 1))
        for s in range(2 * D):
            ax, hi = s // 2, s % 2
            n_neu += m["kind"][s] == 1 and types[s] == 1
            tang = [x for x in range(D) if x != ax]
            for cc in itertools.product(range(1, N + 1), repeat=D - 1):
                pos = [0] * D
                for k, tt in enumerate(tang):
                    pos[tt] = cc[k]
                pos[ax] = N + 1 if hi else 0
                x = np.array([lo[i] + (pos[i] - 0.5) * h for i in range(D)])
                assert abs(_g(a, D, pos) - lin(x)) < 1e-13
    assert n_neu > 0


@pytest.mark.parametrize("D,seed", [(2, 61), (3, 62)])
def test_neumann_box_operator_equals_geometric_assembly(D, seed):
    """With Neumann sides the box machinery still applies exactly the
    geometrically assembled composite operator (Neumann face: +1/h^2 on the
    diagonal instead of -1/h^2, datum weight 1/h instead of 2/h^2), and so do
    the explicit rows."""
    t = random_amr(D, 4, 2, 2, seed)
    t.set_boundary_types(TYPES[D])
    e = t.export()
    K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], TYPES[D])
    rng = np.random.default_rng(seed)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    ref = K @ u + B @ b
    assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(t.leaf_rows() - K).max() <= 1e-12 * abs(K).max()


@pytest.mark.parametrize("D,seed", [(2, 63), (3, 64)])
def test_neumann_discrete_divergence_theorem(D, seed):
    """Sec. 3.3 conservation with Neumann sides: the volume integral of A(u)
    equals the boundary flux sum, where a Neumann face contributes its
    prescribed flux area * b exactly:
    sum h^D (A u)_i = sum_Dirichlet h^(D-2) (2 b - 2 u_i) + sum_Neumann h^(D-1) b."""
    types = TYPES[D]
    t = random_amr(D, 4, 2, 2, seed)
    t.set_boundary_types(types)
    e = t.export()
    rng = np.random.default_rng(seed)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    vol = composite.cell_volumes(D, 4, e["level"], e["children"])
    _, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types)
    area = composite.face_areas(D, 4, e["level"], e["idx"], e["children"])
    h_f = area ** (1.0 / (D - 1))
    cell_of_face = np.asarray(abs(B).tocsc().argmax(axis=0)).ravel()
    _, side = face_sides(t)
    neu = np.array([types[s] == 1 for s in side])
    flux = np.where(neu, h_f ** (D - 1) * b, h_f ** (D - 2) * (2 * b - 2 * u[cell_of_face]))
    assert neu.any() and (~neu).any()
    assert abs(np.sum(vol * Au) - np.sum(flux)) <= 1e-12 * np.sum(np.abs(vol * Au))


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 2, 65), (3, 4, 1, 2, 66)])
def test_neumann_multigrid_converges_to_dense_solution(D, N, uni, extra, seed):
    """FAS multigrid with mixed Dirichlet/Neumann sides converges to the
    direct sparse solve of the composite system."""
    t = random_amr(D, N, uni, extra, seed, frac=0.4)
    t.set_boundary_types(TYPES[D])
    e = t.export()
    K, B = composite.assemble(D, N, e["level"], e["idx"], e["children"], TYPES[D])
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    ref = spla.spsolve(K.tocsc(), rho - B @ b)
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.zero_solution()
    t.solve(1e-13, 80)
    u = t.get_solution()
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


def test_neumann_second_order_discretisation_error():
    """u = exp(x) sin(2y) + x^2 on [0,1]^2, Neumann (inhomogeneous) at x = 0
    and x = 1, Dirichlet at y = 0 and y = 1: the max error drops by about 4
    per halving of h."""
    u = lambda x: np.exp(x[..., 0]) * np.sin(2 * x[..., 1]) + x[..., 0] ** 2
    grad = lambda x: np.array([np.exp(x[0]) * np.sin(2 * x[1]) + 2 * x[0], 2 * np.exp(x[0]) * np.cos(2 * x[1])])
    lap = lambda x: -3 * np.exp(x[..., 0]) * np.sin(2 * x[..., 1]) + 2
    types = [1, 1, 0, 0]
    errs = []
    for lvl in (3, 4, 5):
        t = OracleTree(2, 8, lvl)
        t.refine_uniform(lvl)
        t.set_boundary_types(types)
        xc = t.cell_centers()
        t.set_rhs(lap(xc))
        t.set_dirichlet(boundary_data(t, types, u, grad))
        t.zero_solution()
        t.solve(1e-12, 60)
        errs.append(np.abs(t.get_solution() - u(xc)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders


def test_invalid_side_types_are_refused():
    """Periodic sides come in pairs (singular problems without a Dirichlet
    side are pinned in test_oracle_singular.py)."""
    t = OracleTree(2, 4, 3)
    t.refine_uniform(2)
    with pytest.raises(ValueError):
        t.set_boundary_types([0, 2, 0, 0])
