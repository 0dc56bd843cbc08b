"""Pins of the oracle's singular problems: only Neumann and periodic sides
(arXiv:1701.04329 Sec. 2-3 allow them; Sec. 4.4's gravity problem subtracts
the mean source).  Reading: the oracle solves A u = rho - c, c making the
source compatible (sum h^D (rho - c) = sum over Neumann faces h^(D-1) b),
and returns the solution of zero volume-weighted mean.  No GPU.

Pins: the bordered dense solve [K w; w^T 0] of the composite system with
the test's own compatibility constant (geometry from the exported tree);
a constant added to rho changes nothing; second-order error for periodic
and for pure-Neumann manufactured solutions."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree
from tests.test_oracle_periodic import random_periodic


def geometry(t):
    """Cell volumes (canonical leaf order) and boundary face areas (canonical
    face order) from the exported tree alone."""
    e = t.export()
    D, N = t.D, t.N
    leaves = np.nonzero(e["children"][:, 0] < 0)[0]
    vols, areas = [], []
    for bx in leaves:
        h = 1.0 / (N * 2.0 ** (e["level"][bx] - 1))
        vols.append(np.full(N ** D, h ** D))
        for s in range(2 * D):
            a, hi = s // 2, s % 2
            off = [0] * D
            off[a] = 1 if hi else -1
            # direction index: lexicographic (z, y, x), x fastest, centre skipped
            idx = sum((off[k] + 1) * 3 ** k for k in range(D))
            centre = (3 ** D - 1) // 2
            d = idx - 1 if idx > centre else idx
            if e["neighbours"][bx][d] == -2:
                areas.append(np.full(N ** (D - 1), h ** (D - 1)))
    return e, np.concatenate(vols), (np.concatenate(areas) if areas else np.zeros(0))


def neumann_mask(t, types):
    xyz = t.face_centers()
    side = np.full(len(xyz), -1)
    for a in range(t.D):
        side[xyz[:, a] == 0.0] = 2 * a
        side[xyz[:, a] == 1.0] = 2 * a + 1
    return np.array([types[s] == 1 for s in side], dtype=bool)


def dense_mean_zero(K, w, rhs):
    n = K.shape[0]
    Kb = sp.bmat([[K, sp.csr_matrix(w.reshape(-1, 1))], [sp.csr_matrix(w.reshape(1, -1)), None]]).tocsc()
    x = spla.spsolve(Kb, np.concatenate([rhs, [0.0]]))
    return x[:n], x[n]


@pytest.mark.parametrize("D,types,seed", [(2, [1, 1, 1, 1], 1), (2, [2, 2, 2, 2], 2), (2, [2, 2, 1, 1], 3),
                                          (3, [1, 1, 1, 1, 1, 1], 4), (3, [2, 2, 2, 2, 1, 1], 5)])
def test_singular_multigrid_equals_bordered_dense_solve(D, types, seed):
    t = random_periodic(D, 4, 2 if D == 2 else 1, 2, seed, types, frac=0.4)
    e, vol, area = geometry(t)
    K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"], types)
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=t.n_leaf_cells) + 3.0
    b = rng.normal(size=t.n_bfaces)
    neu = neumann_mask(t, types) if len(b) else np.zeros(0, bool)
    c = (np.sum(vol * rho) - np.sum(area[neu] * b[neu])) / np.sum(vol)
    ref, lam = dense_mean_zero(K, vol, (rho - c) - B @ b)
    assert abs(lam) <= 1e-8 * np.abs(ref).max()  # compatible: the border multiplier vanishes
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.zero_solution()
    hist = []
    t.solve(1e-11, 80, history=hist)
    u = t.get_solution()
    assert hist[-1] <= 1e-11
    assert abs(np.sum(vol * u)) <= 1e-12 * np.abs(u).max()
    assert np.abs(u - ref).max() <= 1e-9 * np.abs(ref).max()


def test_constant_in_the_source_changes_nothing():
    t = random_periodic(2, 8, 2, 1, 7, [2, 2, 1, 1], frac=0.4)
    x = t.cell_centers()
    rho = np.sin(6 * x[:, 0]) + x[:, 1]
    b = np.cos(3 * t.face_centers()[:, 0])
    sols = []
    for k in (0.0, 5.0):
        t.set_rhs(rho + k)
        t.set_dirichlet(b)
        t.zero_solution()
        t.solve(1e-12, 80)
        sols.append(t.get_solution())
    assert np.abs(sols[0] - sols[1]).max() <= 1e-10 * np.abs(sols[0]).max()


@pytest.mark.parametrize("types,u,lap", [
    ([2, 2, 2, 2], lambda x: np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1]),
     lambda x: -8 * np.pi ** 2 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])),
    ([1, 1, 1, 1], lambda x: np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]),
     lambda x: -2 * np.pi ** 2 * np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]))])
def test_singular_second_order_discretisation_error(types, u, lap):
    """Zero-mean manufactured solutions (periodic; zero normal derivative):
    the error falls by about 4 per halving of h."""
    errs = []
    for lvl in (3, 4, 5):
        t = OracleTree(2, 8, lvl)
        t.set_boundary_types(types)
        t.refine_uniform(lvl)
        xc = t.cell_centers()
        t.set_rhs(lap(xc))
        t.set_dirichlet(np.zeros(t.n_bfaces))
        t.zero_solution()
        t.solve(1e-12, 60)
        errs.append(np.abs(t.get_solution() - u(xc)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (orders, errs)


def test_singular_with_variable_coefficients_is_refused():
    t = OracleTree(2, 4, 3)
    t.set_boundary_types([1, 1, 1, 1])
    with pytest.raises(Exception):
        t.set_operator(1)
