"""Pins of the CPU oracle against what the paper and the mathematics fix
(arXiv:1701.04329).  No GPU.  Each test names the passage it checks."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import workloads as W
from tests.treecheck import check_tree

RNG = np.random.default_rng(12345)


def random_amr(D, N, uniform, extra, seed, frac=0.3, n_buf=0, deref_rounds=0):
    """A tree refined at random places (Sec. 2.3 rules), optionally followed
    by derefinement rounds."""
    rng = np.random.default_rng(seed)
    t = OracleTree(D, N, uniform + extra)
    t.refine_uniform(uniform)
    for _ in range(extra):
        nl = t.nleaf
        pick = rng.random(nl) < frac
        flags = np.repeat(pick.astype(np.int8), N ** D)
        t.adapt(flags, n_buf)
    for _ in range(deref_rounds):
        nl = t.nleaf
        pick = rng.random(nl) < 0.7
        flags = -np.repeat(pick.astype(np.int8), N ** D)
        t.adapt(flags, n_buf)
    return t


# ---------------------------------------------------------------- tree (Sec. 2.1-2.3)

@pytest.mark.parametrize("D", [2, 3])
def test_uniform_box_counts(D):
    """Sec. 1.3: refining a box adds 2^D children; a uniform tree to level l
    holds 2^(D(l-1)) boxes on level l."""
    t = OracleTree(D, 4, 5)
    t.refine_uniform(4 if D == 2 else 3)
    lv = t.export()["level"]
    for l in range(1, lv.max() + 1):
        assert (lv == l).sum() == 2 ** (D * (l - 1))


@pytest.mark.parametrize("D,seed", [(2, 1), (2, 2), (3, 3), (3, 4)])
def test_tree_invariants_random_adapt(D, seed):
    """Sec. 2.1-2.3: parent/children/neighbour ids follow from the spatial
    indices, neighbours are reciprocal, boxes are fully refined or not at
    all, 2:1 balance holds across faces, edges and corners, leaves tile the
    domain, and boxes stay Morton-sorted per level -- also after derefinement."""
    t = random_amr(D, 4, 2, 3 if D == 2 else 2, seed, n_buf=1, deref_rounds=2)
    check_tree(t.export(), D)


def test_adapt_one_level_per_call_and_buffer():
    """Sec. 2.3: one adaptation changes the level by at most one; cells within
    N_buf cells of a flagged cell also refine the (diagonal) neighbour."""
    t = OracleTree(2, 8, 6)
    t.refine_uniform(2)  # 2x2 boxes
    flags = np.zeros(t.n_leaf_cells, np.int8)
    # leaf 0 is box (1,1); flag its cell (8,8) (0-based 7,7): near +x, +y and the diagonal
    flags[0 * 64 + 7 * 8 + 7] = 1
    added, removed = t.adapt(flags, 2)
    e = t.export()
    assert e["level"].max() == 3
    assert added == 16 and removed == 0  # all four level-2 boxes refined (buffer incl. diagonal)
    t2 = OracleTree(2, 8, 6)
    t2.refine_uniform(2)
    flags[:] = 0
    flags[0 * 64 + 3 * 8 + 3] = 1  # interior cell: no buffer reach
    assert t2.adapt(flags, 2) == (4, 0)


def test_derefine_respects_balance():
    """Sec. 2.3: children are removed only if all are flagged and 2:1 stays."""
    t = OracleTree(2, 4, 5)
    t.refine_uniform(3)
    a, r = t.adapt(-np.ones(t.n_leaf_cells, np.int8), 0)
    assert r == 16 and a == 0  # every level-3 box removed
    check_tree(t.export(), 2)


# ---------------------------------------------------------------- ghost cells (Sec. 2.4, 3.3)

def _cf_tree(D, N=4):
    """Uniform level 2 with one box refined once more: level-3 boxes meet
    level-2 leaves across refinement boundaries."""
    t = OracleTree(D, N, 3)
    t.refine_uniform(2)
    flags = np.zeros(t.n_leaf_cells, np.int8)
    flags[: N ** D] = 1  # leaf 0
    t.adapt(flags, 0)
    return t


def _set_all(t, fn):
    """Set u on every multigrid box interior from fn(x) at cell centres."""
    boxes = t.mg_boxes()
    e = t.export()
    for b, m in enumerate(boxes):
        M = m["M"]
        D = t.D
        if m["tbox"] >= 0:
            lo = (e["idx"][m["tbox"]] - 1) / 2.0 ** (m["level"] - 1)
        else:
            lo = np.zeros(D)
        h = 1.0 / (M * 2.0 ** (m["level"] - 1)) if m["tbox"] >= 0 else 1.0 / M
        a = np.zeros((M + 2,) * D)
        for c in itertools.product(range(M), repeat=D):
            x = np.array([lo[ax] + (c[ax] + 0.5) * h for ax in range(D)])
            a[tuple(c[::-1][i] + 1 for i in range(D))] = fn(x)
        t.mg_set(b, 0, a)
    return boxes


def _g(a, D, pos):
    """ghosted array access with pos in (x, y[, z]) order"""
    return a[tuple(pos[::-1])]


@pytest.mark.parametrize("D", [2, 3])
def test_refinement_ghosts_conservative(D):
    """Sec. 3.3, Eq. mg-gc-condition: the ghost values under one coarse face
    cell satisfy the flux-conservation constraint (2D: g1 + g2 = u_H +
    3/4(u_31 + u_32) - 1/4(u_41 + u_42); 3D: the four ghosts sum to
    2 u_H + 3/4 sum u_inner - 1/4 sum u_second)."""
    N = 4
    t = _cf_tree(D, N)
    rng = np.random.default_rng(7)
    boxes = _set_all(t, lambda x: rng.normal())
    t.fill_ghosts(3, 0)
    checked = 0
    for b, m in enumerate(boxes):
        if m["level"] != 3:
            continue
        a = t.mg_get(b, 0, N)
        for s in range(2 * D):
            if m["kind"][s] != 2:
                continue
            q = m["nbid"][s]
            cq = t.mg_get(q, 0, N)
            ax, hi = s // 2, s % 2
            tang = [x for x in range(D) if x != ax]
            ghost, inner, second = (N + 1, N, N - 1) if hi else (0, 1, 2)
            for cc in itertools.product(range(N // 2), repeat=D - 1):
                g = inner_s = second_s = 0.0
                for fc in itertools.product((0, 1), repeat=D - 1):
                    pos = [0] * D
                    for k, tt in enumerate(tang):
                        pos[tt] = 2 * cc[k] + fc[k] + 1
                    p = list(pos); p[ax] = ghost; g += _g(a, D, p)
                    p = list(pos); p[ax] = inner; inner_s += _g(a, D, p)
                    p = list(pos); p[ax] = second; second_s += _g(a, D, p)
                cpos = [0] * D
                cpos[ax] = 1 if hi else N
                for k, tt in enumerate(tang):
                    cpos[tt] = m["poff"][tt] + cc[k] + 1
                uH = _g(cq, D, cpos)
                want = 2 ** (D - 2) * uH + 0.75 * inner_s - 0.25 * second_s
                assert abs(g - want) <= 1e-13 * (1 + abs(want))
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("D", [2, 3])
def test_ghosts_exact_for_linear_fields(D):
    """Sec. 3.3 scheme and the Dirichlet ghost 2b - u reproduce a linear
    field exactly at the ghost centres (they are linear extrapolations);
    constants are reproduced bit for bit."""
    N = 4
    t = _cf_tree(D, N)
    coef = np.array([0.3, -1.7, 0.9][:D])
    lin = lambda x: 0.25 + x @ coef
    t.set_dirichlet(lin(t.face_centers()))
    boxes = _set_all(t, lin)
    e = t.export()
    for lvl in (1, 2, 3):
        t.fill_ghosts(lvl, 0)
    for b, m in enumerate(boxes):
        if m["tbox"] < 0:
            continue
        a = t.mg_get(b, 0, N)
        lo = (e["idx"][m["tbox"]] - 1) / 2.0 ** (m["level"] - 1)
        h = 1.0 / (N * 2.0 ** (m["level"] - 1))
        for s in range(2 * D):
            ax, hi = s // 2, s % 2
            tang = [x for x in range(D) if x != ax]
            for cc in itertools.product(range(1, N + 1), repeat=D - 1):
                pos = [0] * D
                for k, tt in enumerate(tang):
                    pos[tt] = cc[k]
                pos[ax] = N + 1 if hi else 0
                x = np.array([lo[i] + (pos[i] - 0.5) * h for i in range(D)])
                assert abs(_g(a, D, pos) - lin(x)) < 1e-13
    # constants, bit for bit
    t.set_dirichlet(np.full(t.n_bfaces, 3.0))
    boxes = _set_all(t, lambda x: 3.0)
    for lvl in (1, 2, 3):
        t.fill_ghosts(lvl, 0)
    for b, m in enumerate(boxes):
        if m["tbox"] >= 0:
            a = t.mg_get(b, 0, N)
            faces = [a[(slice(1, N + 1),) * i + (g,) + (slice(1, N + 1),) * (D - 1 - i)]
                     for i in range(D) for g in (0, N + 1)]
            assert all(np.all(f == 3.0) for f in faces)


# ---------------------------------------------------------------- prolongation / restriction (Sec. 2.5)

@pytest.mark.parametrize("D", [2, 3])
def test_prolongation_exact_for_linear_and_restriction_of_constants(D):
    """Sec. 2.5: the 2-1-1 / 1-1-1-1 schemes are linear interpolations (exact
    for linear fields away from the boundary ghosts); averaging restriction
    of a constant is that constant."""
    N = 8
    t = OracleTree(D, N, 3)
    t.refine_uniform(2)
    t.zero_solution()
    coef = np.array([0.7, -0.4, 1.1][:D])
    lin = lambda x: 2.0 + x @ coef
    boxes = _set_all(t, lin)
    for b, m in enumerate(boxes):
        if m["level"] == 2:
            t.mg_set(b, 0, np.zeros((N + 2,) * D))  # fine u = 0, coarse u = lin, vold = 0
    t.correct(2)
    e = t.export()
    for b, m in enumerate(boxes):
        if m["level"] != 2:
            continue
        a = t.mg_get(b, 0, N)
        lo = (e["idx"][m["tbox"]] - 1) / 2.0
        h = 1.0 / (2 * N)
        for c in itertools.product(range(N), repeat=D):
            x = np.array([lo[i] + (c[i] + 0.5) * h for i in range(D)])
            if np.any(x < 1.5 / N) or np.any(x > 1 - 1.5 / N):
                continue  # stencil reaches the homogeneous boundary ghost
            assert abs(_g(a, D, [ci + 1 for ci in c]) - lin(x)) < 1e-13
    # restriction of a constant
    boxes = _set_all(t, lambda x: 0.3)
    t.restrict(2, 0)
    a = t.mg_get([i for i, m in enumerate(boxes) if m["level"] == 1][0], 0, N)
    assert np.all(a[(slice(1, N + 1),) * D] == 0.3)


# ---------------------------------------------------------------- GSRB (Sec. 3.1)

def test_gsrb_red_update_solves_locally():
    """Sec. 3.1: after a red half-sweep each interior red cell locally solves
    the 5-point equation with its (unchanged) black neighbours."""
    N = 8
    t = OracleTree(2, N, 1)
    rng = np.random.default_rng(3)
    t.set_rhs(rng.normal(size=t.n_leaf_cells))
    t.set_dirichlet(rng.normal(size=t.n_bfaces))
    t.set_solution(rng.normal(size=t.n_leaf_cells))
    t.fill_ghosts(1, 0)
    t.gsrb_half(1, 0)
    b = [i for i, m in enumerate(t.mg_boxes()) if m["level"] == 1][0]
    u = t.mg_get(b, 0, N)
    rho = t.mg_get(b, 1, N)
    h = 1.0 / N
    for j in range(2, N):
        for i in range(2, N):
            if (i + j) % 2:
                continue
            r = rho[j, i] - (u[j, i - 1] + u[j, i + 1] + u[j - 1, i] + u[j + 1, i] - 4 * u[j, i]) / h ** 2
            assert abs(r) < 1e-12 * (1 + abs(rho[j, i]))


def test_gsrb_independent_of_box_decomposition():
    """The smoother acts box by box but ghosts are refilled before every
    half-sweep, so a 32^2 grid of 1 box (N=32), 4 boxes (N=16) or 16 boxes
    (N=8) gives identical values after several sweeps (bit for bit)."""
    outs = []
    for N, lvl in ((32, 1), (16, 2), (8, 3)):
        t = OracleTree(2, N, lvl)
        t.refine_uniform(lvl)
        x = t.cell_centers()
        xf = t.face_centers()
        t.set_rhs(np.sin(7 * x[:, 0]) * np.cos(5 * x[:, 1]))
        t.set_dirichlet(np.cos(3 * xf[:, 0] + xf[:, 1]))
        t.zero_solution()
        t.smooth(lvl, 3)
        u = t.get_solution()
        # canonical order -> global (x, y) grid
        e = t.export()
        g = np.zeros((32, 32))
        leaves = np.nonzero(e["children"][:, 0] < 0)[0]
        for li, b in enumerate(leaves):
            i0, j0 = (e["idx"][b] - 1) * N
            g[j0:j0 + N, i0:i0 + N] = u[li * N * N:(li + 1) * N * N].reshape(N, N)
        outs.append(g)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_gsrb_converges_to_five_point_solution():
    """Gauss-Seidel converges to the solution of the standard 5-point system
    (Dirichlet via 2b - u), here built with scipy's kron of 1D stencils."""
    N = 16
    t = OracleTree(2, N, 1)
    x = t.cell_centers()
    rho = np.sin(3 * x[:, 0]) + x[:, 1]
    t.set_rhs(rho)
    t.set_dirichlet(np.zeros(t.n_bfaces))
    t.zero_solution()
    t.smooth(1, 3000)
    h = 1.0 / N
    T = sp.diags([np.ones(N - 1), -2 * np.ones(N), np.ones(N - 1)], [-1, 0, 1]).tolil()
    T[0, 0] = T[N - 1, N - 1] = -3.0  # ghost 2*0 - u
    I = sp.identity(N)
    A = (sp.kron(I, T) + sp.kron(T, I)) / h ** 2
    ref = spla.spsolve(A.tocsc(), rho)
    assert np.abs(t.get_solution() - ref).max() < 1e-10 * np.abs(ref).max()


# ---------------------------------------------------------------- composite operator (Sec. 3.2-3.3)

@pytest.mark.parametrize("D,seed", [(2, 11), (2, 12), (3, 13)])
def test_box_operator_equals_geometric_assembly(D, seed):
    """The box machinery (restriction to parents, ghost fill, stencil) applies
    exactly the composite operator assembled geometrically from (level,
    global cell index) lookups, and so do the oracle's explicit rows."""
    t = random_amr(D, 4, 2, 2, seed)
    assert any(2 in m["kind"] for m in t.mg_boxes())  # has refinement boundaries
    e = t.export()
    K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"])
    rng = np.random.default_rng(seed)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    ref = K @ u + B @ b
    assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()
    Kr = t.leaf_rows()
    assert abs(Kr - K).max() <= 1e-12 * abs(K).max()


@pytest.mark.parametrize("D,seed", [(2, 21), (3, 22)])
def test_discrete_divergence_theorem(D, seed):
    """Sec. 3.3: with conservative refinement-boundary ghosts the volume
    integral of A(u) equals the boundary flux sum, for any u and b:
    sum_leaves h^D (A u)_i = sum_faces h^(D-2) (2 b_f - 2 u_i(f))."""
    t = random_amr(D, 4, 2, 2, seed)
    assert any(2 in m["kind"] for m in t.mg_boxes())
    e = t.export()
    rng = np.random.default_rng(seed)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    vol = composite.cell_volumes(D, 4, e["level"], e["children"])
    lhs = np.sum(vol * Au)
    _, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"])
    area = composite.face_areas(D, 4, e["level"], e["idx"], e["children"])
    h_f = area ** (1.0 / (D - 1))
    cell_of_face = np.asarray(B.tocsc().argmax(axis=0)).ravel()
    rhs = np.sum(h_f ** (D - 2) * (2 * b - 2 * u[cell_of_face]))
    scale = np.sum(np.abs(vol * Au))
    assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 2, 31), (2, 4, 1, 3, 32), (3, 4, 1, 2, 33)])
def test_multigrid_converges_to_dense_solution(D, N, uni, extra, seed):
    """FAS multigrid on the tree converges to the unique solution of the
    composite leaf system (direct sparse solve on tiny trees)."""
    t = random_amr(D, N, uni, extra, seed, frac=0.4)
    e = t.export()
    K, B = composite.assemble(D, N, e["level"], e["idx"], e["children"])
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    ref = spla.spsolve(K.tocsc(), rho - B @ b)
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.zero_solution()
    t.solve(1e-13, 60)
    u = t.get_solution()
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


# ---------------------------------------------------------------- convergence (Sec. 4.1)

def _solve_problem(p, tol=1e-11):
    t = OracleTree(p.dim, p.box_n, p.max_level)
    p.build(t)
    rho, b = p.data(t)
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.zero_solution()
    return t, t.solve(tol, 60)


def test_second_order_discretisation_error():
    """Second-order accuracy: the max error against the manufactured solution
    drops by ~4 per halving of h (uniform grids and the AMR grid refined one
    level everywhere)."""
    errs = []
    for lvl in (3, 4, 5):
        p = W.gauss2d(uniform_level=lvl, max_level=lvl, s=0.2)
        t, _ = _solve_problem(p)
        errs.append(np.abs(t.get_solution() - p.u_exact(t.cell_centers())).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders
    # AMR: gauss2d tree, then every leaf split once
    p = W.gauss2d(max_level=6)
    t, _ = _solve_problem(p)
    e1 = np.abs(t.get_solution() - p.u_exact(t.cell_centers())).max()
    p2 = W.gauss2d(max_level=7)
    t2 = OracleTree(2, 8, 7)
    p2.build  # same criterion; split every leaf of the level-6 tree instead
    t2.refine_uniform(4)
    W.adapt_until_stable(t2, lambda x, h, lv: (np.abs(p.rho(x)) * h ** 2 > 1e-4).astype(np.int8) * (lv < 6))
    t2.adapt(np.ones(t2.n_leaf_cells, np.int8), 0)
    rho, b = p2.data(t2)
    t2.set_rhs(rho); t2.set_dirichlet(b); t2.zero_solution(); t2.solve(1e-11, 60)
    e2 = np.abs(t2.get_solution() - p2.u_exact(t2.cell_centers())).max()
    assert np.log2(e1 / e2) > 1.5, (e1, e2)


def test_second_order_discretisation_error_3d():
    """The 3D manufactured twin of the benchmark workload (the two Gaussians
    of opposite sign as the exact solution, its Laplacian as the source, its
    face values as Dirichlet data): the max error drops by ~4 per halving of
    h on uniform 16^3 / 32^3 / 64^3 grids (orders 1.86, 1.98 measured), and
    by ~4 when every leaf of a refined tree is split once (1.94)."""
    errs = []
    for lvl in (2, 3, 4):
        p = W.twin3d(uniform_level=lvl, extra_levels=0, s=0.15)
        t, _ = _solve_problem(p)
        errs.append(np.abs(t.get_solution() - p.u_exact(t.cell_centers())).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders
    p = W.twin3d(uniform_level=2, extra_levels=2, s=0.15, frac=0.3)
    t, _ = _solve_problem(p)
    assert len(set(t.leaf_levels())) > 1
    e1 = np.abs(t.get_solution() - p.u_exact(t.cell_centers())).max()
    t2 = OracleTree(3, 8, 5)
    p.build(t2)
    t2.adapt(np.ones(t2.n_leaf_cells, np.int8), 0)
    rho, b = p.data(t2)
    t2.set_rhs(rho); t2.set_dirichlet(b); t2.zero_solution(); t2.solve(1e-11, 60)
    e2 = np.abs(t2.get_solution() - p.u_exact(t2.cell_centers())).max()
    assert np.log2(e1 / e2) > 1.5, (e1, e2)


def test_one_fmg_reaches_discretisation_error_and_cycle_factors():
    """Sec. 4.1: one FMG cycle gives convergence up to the discretisation
    error, and each further FMG cycle reduces the residual by a factor of
    about 0.07 (here the asymptotic factor must lie in [0.02, 0.1])."""
    p = W.gauss2d()
    t = OracleTree(2, 8, p.max_level)
    p.build(t)
    rho, b = p.data(t)
    t.set_rhs(rho); t.set_dirichlet(b); t.zero_solution()
    ue = p.u_exact(t.cell_centers())
    t.fmg()
    e_fmg = np.abs(t.get_solution() - ue).max()
    hist = []
    for _ in range(5):
        t.fmg()
        r, pm = t.residual_norm()
        hist.append(r / pm)
    e_conv = np.abs(t.get_solution() - ue).max()
    assert e_fmg <= 2.0 * e_conv
    f = hist[-1] / hist[-2]
    assert 0.02 <= f <= 0.1, hist
    # V-cycles: recorded per-cycle reduction, asserted loosely
    t.zero_solution()
    hist = []
    t.solve(1e-10, 30, history=hist)
    factors = np.array(hist[1:]) / np.array(hist[:-1])
    assert factors.max() < 0.15, factors
