"""Pins of the oracle's edge/corner ghost cells and prolongation schemes
(arXiv:1701.04329 Sec. 2.4: corner ghosts copied from a diagonal neighbour
or linearly extrapolated, b + c - a; Sec. 2.5: bilinear / trilinear, the
linear (1/2,1/4,1/4) / (1/4,1/4,1/4,1/4) and zeroth-order prolongation).
No GPU.

Pins: every ghost cell (side, edge, corner; same-level, refinement-boundary
and domain-boundary ones) of every box reproduces a linear field exactly;
corner ghosts equal the diagonal neighbour's cells where it exists; with the
extrapolated corner, bilinear interpolation through (a,b,c,d) is the linear
interpolation through (a,b,c) (the property Sec. 2.4 points out), so the
bilinear correction reproduces linear fields everywhere and bilinear fields
inside; the zeroth-order one copies; every scheme converges to the same
dense composite solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import composite
from oracle.oracle import OracleTree


def amr(D, N, uniform, extra, seed, frac=0.35):
    rng = np.random.default_rng(seed)
    t = OracleTree(D, N, uniform + extra)
    t.refine_uniform(uniform)
    for _ in range(extra):
        t.adapt(np.repeat((rng.random(t.nleaf) < frac).astype(np.int8), N ** D), 1)
    return t


def centres(D, M, h, x0):
    """cell centres of a ghosted M-box, array [k][j][i][axis] (3D) or [j][i][axis]"""
    g = (np.arange(M + 2) - 0.5) * h
    if D == 2:
        Y, X = np.meshgrid(g + x0[1], g + x0[0], indexing="ij")
        return np.stack([X, Y], -1)
    Z, Y, X = np.meshgrid(g + x0[2], g + x0[1], g + x0[0], indexing="ij")
    return np.stack([X, Y, Z], -1)


def box_origin(t, e, m):
    """lower corner of a multigrid box: from its tree box, or the unit root below level 1"""
    if m["tbox"] < 0:
        return np.zeros(t.D), 1.0 / m["M"]
    h = 1.0 / (t.N * 2 ** (m["level"] - 1))
    return (e["idx"][m["tbox"]] - 1) * t.N * h, h


@pytest.mark.parametrize("D,seed", [(2, 401), (3, 402)])
def test_all_ghosts_reproduce_a_linear_field(D, seed):
    t = amr(D, 4, 2 if D == 2 else 1, 2, seed)
    coef = np.array([0.3, -1.2, 0.7][:D])

    def f(x):
        return 0.25 + x @ coef
    t.set_rhs(np.zeros(t.n_leaf_cells))
    t.set_dirichlet(f(t.face_centers()))
    e = t.export()
    mg = t.mg_boxes()
    for b, m in enumerate(mg):               # the field on every box of every level
        x0, h = box_origin(t, e, m)
        t.mg_set(b, 0, f(centres(D, m["M"], h, x0)))
    for l in range(t.lmin, t.highest_level + 1):
        t.fill_ghosts(l, 0)
        t.fill_corner_ghosts(l, 0)
    worst = 0.0
    for b, m in enumerate(mg):
        x0, h = box_origin(t, e, m)
        want = f(centres(D, m["M"], h, x0))
        got = t.mg_get(b, 0, m["M"])
        worst = max(worst, np.abs(got - want).max())
    assert worst <= 1e-13


@pytest.mark.parametrize("D", [2, 3])
def test_corner_ghosts_copy_the_diagonal_neighbour(D):
    t = OracleTree(D, 4, 3)
    t.refine_uniform(3 if D == 2 else 2)
    rng = np.random.default_rng(5)
    t.set_rhs(np.zeros(t.n_leaf_cells))
    t.set_dirichlet(rng.normal(size=t.n_bfaces))
    t.set_solution(rng.normal(size=t.n_leaf_cells))
    L = t.highest_level
    t.fill_ghosts(L, 0)
    t.fill_corner_ghosts(L, 0)
    e = t.export()
    mg = t.mg_boxes()
    pos = {(m["level"],) + tuple(int(v) for v in e["idx"][m["tbox"]]): b for b, m in enumerate(mg) if m["tbox"] >= 0}
    checked = 0
    for b, m in enumerate(mg):
        if m["level"] != L:
            continue
        idx = tuple(int(v) for v in e["idx"][m["tbox"]])
        q = pos.get((L,) + tuple(v - 1 for v in idx))      # the (-1,-1[,-1]) diagonal neighbour
        if q is None:
            continue
        g = t.mg_get(b, 0, 4)
        n = t.mg_get(q, 0, 4)
        assert g[(0,) * D] == n[(4,) * D]
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("D,seed", [(2, 411), (3, 412)])
def test_correction_schemes_on_linear_and_multilinear_fields(D, seed):
    """Prolong a coarse difference d = f (v_H = f, v'_H = 0) to the finest
    boxes: linear f is reproduced by the linear and bi/trilinear schemes, the
    product f = x y (z) by bi/trilinear, at every fine cell off the
    outermost layer (there the coarse ghosts are -d: the correction vanishes
    on a Dirichlet side); zeroth order adds the coarse value everywhere."""
    t = OracleTree(D, 4, 3)
    t.refine_uniform(3 if D == 2 else 2)
    L = t.highest_level
    t.set_rhs(np.zeros(t.n_leaf_cells))
    t.set_homogeneous(1)
    e = t.export()
    mg = t.mg_boxes()
    lin = np.array([0.3, -1.2, 0.7][:D])
    for scheme, fun in ((0, lambda x: 0.5 + x @ lin), (1, lambda x: 0.5 + x @ lin),
                        (1, lambda x: np.prod(x, -1)), (2, lambda x: 0.5 + x @ lin)):
        t.set_prolong(scheme)
        for b, m in enumerate(mg):
            x0, h = box_origin(t, e, m)
            c = centres(D, m["M"], h, x0)
            if m["level"] == L - 1:
                t.mg_set(b, 0, fun(c))
                t.mg_set(b, 2, np.zeros_like(c[..., 0]))   # v' = 0, so d = f
            elif m["level"] == L:
                t.mg_set(b, 0, np.zeros_like(c[..., 0]))
        t.correct(L)
        for b, m in enumerate(mg):
            if m["level"] != L:
                continue
            x0, h = box_origin(t, e, m)
            c = centres(D, m["M"], h, x0)
            got = t.mg_get(b, 0, m["M"])[(slice(1, -1),) * D]
            inner = (slice(1, -1),) * D
            want = fun(c)[inner]
            if scheme == 2:                         # zeroth order: the coarse cell's value
                H = 2 * h
                want = fun((np.floor(c[inner] / H) + 0.5) * H)
                assert np.abs(got - want).max() <= 1e-14
            else:                                   # off the outermost layer
                away = np.all((c[inner] > h) & (c[inner] < 1 - h), -1)
                assert away.sum() > 0 and np.abs(got - want)[away].max() <= 1e-14, scheme


def test_bilinear_through_extrapolated_corner_is_linear():
    """Sec. 2.4: with d = b + c - a, bilinear interpolation through
    (a, b, c, d) equals linear interpolation through (a, b, c)."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        a, b, c = rng.normal(size=3)
        d = b + c - a
        s, r = rng.random(2)
        bil = a * (1 - s) * (1 - r) + b * s * (1 - r) + c * (1 - s) * r + d * s * r
        assert abs(bil - (a + (b - a) * s + (c - a) * r)) <= 1e-14


@pytest.mark.parametrize("D,seed", [(2, 421), (3, 422)])
def test_every_scheme_converges_to_the_dense_solution(D, seed):
    t = amr(D, 4, 2 if D == 2 else 1, 2, seed, frac=0.4)
    e = t.export()
    K, B = composite.assemble(D, 4, e["level"], e["idx"], e["children"])
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    ref = spla.spsolve(K.tocsc(), rho - B @ b)
    for scheme in (0, 1, 2):
        t.set_prolong(scheme)
        t.set_rhs(rho)
        t.set_dirichlet(b)
        t.zero_solution()
        t.solve(1e-13, 120)
        assert np.abs(t.get_solution() - ref).max() <= 1e-10 * np.abs(ref).max(), scheme


def test_cycle_factors_by_scheme():
    """2D, 256^2 + one level around a Gaussian: V(2,2) reductions measured
    above the roundoff floor (down to 1e-9): linear 0.065-0.11, bilinear about
    0.09, zeroth order 0.03-0.06 per cycle; the FMG cycle leaves 2.8e-3,
    4.7e-3 and 0.43 (zeroth order interpolates the FMG solution poorly)."""
    out = {}
    for scheme in (0, 1, 2):
        t = OracleTree(2, 8, 6)
        t.refine_uniform(5)
        x = t.cell_centers()
        t.adapt((np.linalg.norm(x - 0.4, axis=1) < 0.2).astype(np.int8), 1)
        x = t.cell_centers()
        t.set_prolong(scheme)
        t.set_rhs(np.exp(-np.sum((x - 0.4) ** 2, 1) / 0.02))
        t.set_dirichlet(np.zeros(t.n_bfaces))
        t.zero_solution()
        hist = []
        t.solve(1e-9, 30, history=hist)
        out[scheme] = (hist[0], max(hist[i + 1] / hist[i] for i in range(len(hist) - 1)))
    assert out[0][0] < 1e-2 and out[1][0] < 1e-2 and out[2][0] > 0.1
    assert out[0][1] <= 0.15 and out[1][1] <= 0.15 and out[2][1] <= 0.15, out
