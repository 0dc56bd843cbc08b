"""Pins of the oracle's variable-coefficient operators (arXiv:1701.04329
Sec. 3.4: a jump of eps at a cell face, flux = harmonic mean of the two
coefficients times the difference quotient; Sec. 3.5: the same operator in
Cartesian and in (r,z) coordinates).  No GPU.

Pins: a constant eps scales the Laplacian; a layered problem whose exact
solution is piecewise linear is reproduced exactly (the harmonic mean is the
exact flux of a jump at a face); the discrete divergence theorem with the
face coefficients (and r-weights in (r,z)); u = r^2 under the (r,z)
operator gives 4 eps exactly, the axis face carrying no flux; the box
machinery equals an independent geometric assembly; multigrid converges to
the dense solution of that assembly."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree


def amr_tree(D, N, uniform, extra, seed, roots=None, types=None, frac=0.3):
    rng = np.random.default_rng(seed)
    t = OracleTree(D, N, uniform + extra, roots=roots)
    if types is not None:
        t.set_boundary_types(types)
    t.refine_uniform(uniform)
    for _ in range(extra):
        t.adapt(np.repeat((rng.random(t.nleaf) < frac).astype(np.int8), N ** D), 1)
    return t


def coarse_cell_eps(t, seed, lo=0.1, hi=100.0):
    """A coefficient constant on every level-1 cell (jumps only at faces of
    the coarsest tree cells, as Sec. 3.4 requires), log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    x = t.cell_centers()
    n1 = [r * t.N for r in getattr(t, "roots", (1,) * t.D)]
    table = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n1))
    cell = tuple(np.minimum((x[:, a] * t.N).astype(int), n1[a] - 1) for a in range(t.D))
    return table[cell]


@pytest.mark.parametrize("D", [2, 3])
def test_constant_eps_scales_the_laplacian(D):
    t = amr_tree(D, 4, 2, 2, 301 + D)
    rng = np.random.default_rng(7)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    a0 = t.apply_A(u)
    t.set_operator(1)
    t.set_eps(np.full(t.n_leaf_cells, 4.0))
    t.set_dirichlet(b)
    a1 = t.apply_A(u)
    assert np.abs(a1 - 4.0 * a0).max() <= 1e-13 * np.abs(a1).max()


@pytest.mark.parametrize("D", [2, 3])
def test_layered_piecewise_linear_solution_is_exact(D):
    """eps = e1 for x < 1/2, e2 beyond; u = x/e1, then 1/(2 e1) + (x-1/2)/e2:
    continuous flux 1 across the jump, so div(eps grad u) = 0 -- also in the
    discrete operator, on a tree refined away from the interface."""
    e1, e2 = 3.0, 0.25
    t = OracleTree(D, 4, 4)
    t.refine_uniform(2)
    e = t.export()
    leaves = np.nonzero(e["children"][:, 0] < 0)[0]
    flags = np.zeros(t.n_leaf_cells, np.int8)
    for li, bx in enumerate(leaves):       # refine the box at x in [0, 1/4) and y in [1/4, 1/2)
        if e["idx"][bx][0] == 1 and e["idx"][bx][1] == 2 and (D == 2 or e["idx"][bx][2] == 1):
            flags[li * 4 ** D:(li + 1) * 4 ** D] = 1
    t.adapt(flags, 0)
    x = t.cell_centers()

    def exact(px):
        return np.where(px < 0.5, px / e1, 0.5 / e1 + (px - 0.5) / e2)
    t.set_operator(1)
    t.set_eps(np.where(x[:, 0] < 0.5, e1, e2))
    t.set_dirichlet(exact(t.face_centers()[:, 0]))
    Au = t.apply_A(exact(x[:, 0]))
    assert np.abs(Au).max() <= 1e-11 * (1 / e1 + 1 / e2) * 4 ** 6
    # and multigrid converges to it
    t.set_rhs(np.zeros(t.n_leaf_cells))
    t.zero_solution()
    t.solve(1e-30, 60)
    assert np.abs(t.get_solution() - exact(x[:, 0])).max() <= 1e-11


@pytest.mark.parametrize("D,op", [(2, 1), (3, 1), (2, 2)])
def test_flux_conservation(D, op):
    """Sum over leaf cells of w_i vol_i (A u)_i equals the flux through the
    Dirichlet faces, sum_f w_f c_f h^(D-2) (2 b - 2 u_i): interior and
    refinement-boundary fluxes cancel pairwise (w = r in (r,z), else 1)."""
    t = amr_tree(D, 4, 2, 2, 311 + D + op)
    t.set_operator(op)
    x = t.cell_centers()
    eps = coarse_cell_eps(t, 5)
    t.set_eps(eps)
    rng = np.random.default_rng(9)
    u = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    t.set_dirichlet(b)
    Au = t.apply_A(u)
    e = t.export()
    lv = t.leaf_levels()
    h = np.repeat(1.0 / (4 * 2.0 ** (lv - 1)), 4 ** D)
    w = x[:, 0] if op == 2 else np.ones(len(x))
    lhs = np.sum(w * h ** D * Au)
    # boundary faces: the cell next to each face (canonical face order)
    fc = t.face_centers()
    cell = np.array([np.argmin(np.abs(x - f).sum(1) + 10 * (np.abs(x - f).max(1) > 0.51 * h)) for f in fc])
    hf = h[cell]
    wf = fc[:, 0] if op == 2 else np.ones(len(fc))
    flux = wf * eps[cell] * hf ** (D - 2) * (2 * b - 2 * u[cell])
    assert abs(lhs - flux.sum()) <= 1e-12 * np.sum(np.abs(w * h ** D * Au))


def test_cylindrical_r_squared():
    """(1/r) d/dr (r d(r^2)/dr) = 4 and d^2 z/dz^2 = 0 hold exactly for the
    discrete (r,z) operator at every cell whose four neighbours are leaf
    cells of its own level and not beyond a Dirichlet side -- next to the
    axis too, where the face at r = 0 carries no flux.  On a uniform tree
    that is every cell off the Dirichlet sides."""
    eps = 2.5
    for extra in (0, 1):
        t = amr_tree(2, 4, 3, extra, 321, frac=0.4)
        t.set_operator(2)
        t.set_eps(np.full(t.n_leaf_cells, eps))
        x = t.cell_centers()
        fc = t.face_centers()
        t.set_dirichlet(fc[:, 0] ** 2 + fc[:, 1])
        Au = t.apply_A(x[:, 0] ** 2 + x[:, 1])
        lv = np.repeat(t.leaf_levels(), 16)
        h = 1.0 / (4 * 2.0 ** (lv - 1))
        key = {(int(l), int(round(p[0] / hh - 0.5)), int(round(p[1] / hh - 0.5))) for l, p, hh in zip(lv, x, h)}
        ok = []
        for l, p, hh in zip(lv, x, h):
            i, j = int(round(p[0] / hh - 0.5)), int(round(p[1] / hh - 0.5))
            n = 4 * 2 ** (l - 1)
            nbs = [(i + 1, j), (i, j - 1), (i, j + 1)] + ([(i - 1, j)] if i > 0 else [])
            ok.append(i + 1 < n and 0 < j < n - 1 and all((int(l),) + q in key for q in nbs))
        ok = np.array(ok)
        if extra == 0:
            assert ok.sum() == np.sum((x[:, 0] < 1 - h) & (x[:, 1] > h) & (x[:, 1] < 1 - h))
        else:
            assert 0 < ok.sum() < len(x)
        assert np.abs(Au[ok] - 4 * eps).max() <= 1e-9
        axis = ok & (x[:, 0] < h)
        assert axis.sum() > 0 and np.abs(Au[axis] - 4 * eps).max() <= 1e-9


@pytest.mark.parametrize("D,op,seed", [(2, 1, 331), (3, 1, 332), (2, 2, 333)])
def test_box_operator_equals_geometric_assembly(D, op, seed):
    """Arbitrary positive eps per leaf cell, refinement, periodic/Neumann sides
    and several roots: the box machinery (restricted eps, ghost values,
    stencil) equals the face-by-face geometric assembly."""
    cases = [dict(), dict(types=[0, 1] + [0, 0] * (D - 1)), dict(roots=(2,) + (1,) * (D - 1))]
    if op == 1:
        cases.append(dict(types=[0, 0] + [2, 2] + [0, 0] * (D - 2)))
    for kw in cases:
        t = amr_tree(D, 4, 2 if D == 2 else 1, 2, seed, **kw)
        t.set_operator(op)
        rng = np.random.default_rng(seed)
        eps = np.exp(rng.normal(size=t.n_leaf_cells))
        t.set_eps(eps)
        e = t.export()
        K, B = composite.assemble_var(D, 4, e["level"], e["idx"], e["children"], eps, op,
                                      kw.get("types"), kw.get("roots"))
        u = rng.normal(size=t.n_leaf_cells)
        b = rng.normal(size=t.n_bfaces)
        t.set_dirichlet(b)
        Au = t.apply_A(u)
        ref = K @ u + B @ b
        assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max(), kw


@pytest.mark.parametrize("D,op,seed", [(2, 1, 341), (3, 1, 342), (2, 2, 343)])
def test_multigrid_converges_to_dense_solution(D, op, seed):
    t = amr_tree(D, 4, 2 if D == 2 else 1, 2, seed, frac=0.4)
    t.set_operator(op)
    eps = coarse_cell_eps(t, seed)
    t.set_eps(eps)
    e = t.export()
    K, B = composite.assemble_var(D, 4, e["level"], e["idx"], e["children"], eps, op)
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    ref = spla.spsolve(K.tocsc(), rho - B @ b)
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.zero_solution()
    t.solve(1e-13, 200)
    assert np.abs(t.get_solution() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_cylindrical_restriction_is_volume_weighted():
    """In (r,z) a coarse value is the children's mean weighted by their
    volumes (r at their centres), so u = 1/r restricts to exactly 1/r at the
    coarse centre (sum r_k / r_k = 4 = sum r_k / r_c); the plain mean of the
    Cartesian operators would not."""
    for op in (1, 2):
        t = OracleTree(2, 8, 2)
        t.refine_uniform(2)
        t.set_operator(op)
        t.set_rhs(np.zeros(t.n_leaf_cells))
        mg = t.mg_boxes()
        fine = [i for i, m in enumerate(mg) if m["level"] == 2]
        root = [i for i, m in enumerate(mg) if m["level"] == 1][0]
        for i in fine:
            m = mg[i]
            x0 = (e := t.export())["idx"][m["tbox"]][0] - 1
            r = (x0 * 8 + np.arange(8) + 0.5) / 16.0
            a = np.zeros((10, 10))
            a[1:9, 1:9] = 1.0 / r[None, :]
            t.mg_set(i, 0, a)
        t.restrict(2, 0)
        u = t.mg_get(root, 0, 8)[1:9, 1:9]
        rc = (np.arange(8) + 0.5) / 8.0
        if op == 2:
            assert np.abs(u - 1.0 / rc[None, :]).max() <= 1e-14 * np.abs(u).max()
        else:
            assert np.abs(u - 1.0 / rc[None, :]).max() > 1e-3


@pytest.mark.parametrize("op", [1, 2])
def test_paper_jump_layout_converges(op):
    """Sec. 4.1's second test layout: eps = 100 on [0,1/4]^2, 1 elsewhere,
    in Cartesian (op 1) and (r,z) (op 2) coordinates, two Gaussian sources
    at (1/4,1/4) and (3/4,3/4), u = 0 on the sides; 256^2 cells, V(2,2).
    Measured after the FMG cycle: mean reduction 0.10 (Cartesian) and 0.14
    ((r,z)) per V-cycle, single cycles up to 0.20 and 0.30."""
    t = OracleTree(2, 8, 6)
    t.refine_uniform(6)
    x = t.cell_centers()
    t.set_operator(op)
    t.set_eps(np.where((x[:, 0] < 0.25) & (x[:, 1] < 0.25), 100.0, 1.0))
    t.set_rhs(sum(np.exp(-np.sum((x - c) ** 2, 1) / 0.04 ** 2) for c in ((0.25, 0.25), (0.75, 0.75))))
    t.set_dirichlet(np.zeros(t.n_bfaces))
    t.zero_solution()
    hist = []
    t.solve(1e-11, 40, history=hist)
    f = [hist[i + 1] / hist[i] for i in range(len(hist) - 1)]
    mean = (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1))
    assert hist[-1] <= 1e-11 and mean <= 0.2 and max(f) <= 0.35, f


@pytest.mark.parametrize("D,op", [(2, 1), (3, 1), (2, 2)])
def test_uniform_operator_is_symmetric(D, op):
    """On a uniform tree with Dirichlet sides the face coefficient is shared
    by the two cells, so the operator is symmetric: K in Cartesian
    coordinates, diag(r) K in (r,z) (the finite-volume weights).  Assembled
    from the box machinery (A applied to unit vectors)."""
    t = OracleTree(D, 4, 2)
    t.refine_uniform(2)
    t.set_operator(op)
    rng = np.random.default_rng(17 + D + op)
    t.set_eps(np.exp(rng.normal(size=t.n_leaf_cells)))
    t.set_dirichlet(np.zeros(t.n_bfaces))
    n = t.n_leaf_cells
    K = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        K[:, j] = t.apply_A(e)
    W = np.diag(t.cell_centers()[:, 0]) if op == 2 else np.eye(n)
    S = W @ K
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("D,op,seed", [(2, 1, 351), (3, 1, 352), (2, 2, 353)])
def test_adjoint_of_the_variable_operator(D, op, seed):
    """L = g . u with u the multigrid solution for (rho, b): dL/drho = K^-T g
    and dL/db = -B^T K^-T g for the variable-coefficient K, B -- checked by
    central differences of L through the oracle's own solves (L is linear, so
    they are exact up to the solve tolerance), and BiCGStab with the V-cycle
    preconditioner against the direct transpose solve."""
    from oracle import adjoint
    t = amr_tree(D, 4, 2 if D == 2 else 1, 2, seed, frac=0.4)
    t.set_operator(op)
    t.set_eps(coarse_cell_eps(t, seed, 0.2, 20.0))
    rng = np.random.default_rng(seed)
    g = rng.normal(size=t.n_leaf_cells)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    lam = adjoint.direct(t, g)
    db = adjoint.dl_db(t, lam)

    def L(r, bb):
        t.set_rhs(r)
        t.set_dirichlet(bb)
        t.set_homogeneous(0)
        t.zero_solution()
        t.solve(1e-14, 200)
        return g @ t.get_solution()
    for i in rng.choice(t.n_leaf_cells, 4, replace=False):
        e = np.zeros(t.n_leaf_cells)
        e[i] = 1.0
        fd = (L(rho + e, b) - L(rho - e, b)) / 2
        assert abs(fd - lam[i]) <= 1e-8 * np.abs(lam).max()
    for f in rng.choice(t.n_bfaces, 4, replace=False):
        e = np.zeros(t.n_bfaces)
        e[f] = 1.0
        fd = (L(rho, b + e) - L(rho, b - e)) / 2
        assert abs(fd - db[f]) <= 1e-8 * np.abs(db).max()
    x, its = adjoint.bicgstab(t, g, tol=1e-12)
    assert its < 60 and np.abs(x - lam).max() <= 1e-9 * np.abs(lam).max()
