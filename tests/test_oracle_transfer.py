"""Pins of the oracle's field transfer on mesh adaptation (arXiv:1701.04329
Sec. 2.3: with prolongation and restriction routines given, they are applied
when boxes are added or removed; Sec. 2.5: the schemes).  No GPU.

Pins: leaves that stay keep their values bit for bit; a derefined parent
gets the mean of its children, so the integral over the domain is conserved
and linear fields stay exact; the linear and bi/trilinear prolongation of a
refined leaf reproduce linear fields (ghosts from the boundary data, the
refinement-boundary scheme and the extrapolated corners); zeroth order
conserves the integral, and refining then derefining returns the field."""
import numpy as np
import pytest

from oracle.oracle import OracleTree

COEF = np.array([0.7, -1.3, 0.4])


def lin(x):
    return 0.25 + x @ COEF[:x.shape[1]]


def volumes(t):
    return np.repeat((1.0 / (t.N * 2.0 ** (t.leaf_levels() - 1))) ** t.D, t.N ** t.D)


def start(D, seed, uniform=2):
    t = OracleTree(D, 4, 6 if D == 2 else 5)
    t.refine_uniform(uniform)
    rng = np.random.default_rng(seed)
    t.adapt(np.repeat((rng.random(t.nleaf) < 0.3).astype(np.int8), 4 ** D), 1)
    return t, rng


@pytest.mark.parametrize("D,scheme", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_refinement_keeps_linear_fields(D, scheme):
    t, rng = start(D, 500 + D + scheme)
    for step in range(2):
        x = t.cell_centers()
        t.set_dirichlet(lin(t.face_centers()))
        flags = np.repeat((rng.random(t.nleaf) < 0.3).astype(np.int8), 4 ** D)
        u, added, removed = t.adapt_transfer(flags, lin(x), 1, scheme)
        assert added > 0
        assert np.abs(u - lin(t.cell_centers())).max() <= 1e-14


@pytest.mark.parametrize("D", [2, 3])
def test_kept_leaves_and_derefinement(D):
    """Random field: leaves that stay are copied exactly; derefinement
    replaces 2^D children by their mean, which conserves sum(vol * u)."""
    t, rng = start(D, 510 + D, uniform=3)
    x = t.cell_centers()
    u = rng.normal(size=t.n_leaf_cells)
    before = {tuple(np.round(c * 4096).astype(int)): v for c, v in zip(x, u)}
    total = np.sum(volumes(t) * u)
    flags = -np.ones(t.n_leaf_cells, np.int8)            # derefine wherever allowed
    v, added, removed = t.adapt_transfer(flags, u, 0, 0)
    assert added == 0 and removed > 0
    assert abs(np.sum(volumes(t) * v) - total) <= 1e-14 * np.sum(volumes(t) * np.abs(v))
    kept = 0
    for c, val in zip(t.cell_centers(), v):
        key = tuple(np.round(c * 4096).astype(int))
        if key in before:
            assert val == before[key]
            kept += 1
    assert 0 < kept < len(v)
    # a linear field stays exact through derefinement
    t2, _ = start(D, 510 + D, uniform=3)
    w, _, _ = t2.adapt_transfer(flags[:t2.n_leaf_cells], lin(t2.cell_centers()), 0, 0)
    assert np.abs(w - lin(t2.cell_centers())).max() <= 1e-14


@pytest.mark.parametrize("D", [2, 3])
def test_zeroth_order_round_trip(D):
    t, rng = start(D, 520 + D)
    u = rng.normal(size=t.n_leaf_cells)
    total = np.sum(volumes(t) * u)
    flags = np.repeat((rng.random(t.nleaf) < 0.4).astype(np.int8), 4 ** D)
    v, added, _ = t.adapt_transfer(flags, u, 0, 2)
    assert added > 0
    assert abs(np.sum(volumes(t) * v) - total) <= 1e-13 * np.sum(volumes(t) * np.abs(v))
    w, _, removed = t.adapt_transfer(-np.ones(t.n_leaf_cells, np.int8), v, 0, 2)
    assert removed >= added
    # every box added above is removed again (nothing else was derefinable before)
    t0, _ = start(D, 520 + D)
    x0 = t0.cell_centers()
    assert t.n_leaf_cells == t0.n_leaf_cells
    ref = {tuple(np.round(c * 4096).astype(int)): val for c, val in zip(x0, u)}
    got = np.array([ref[tuple(np.round(c * 4096).astype(int))] for c in t.cell_centers()])
    assert np.abs(w - got).max() <= 1e-15 * np.abs(u).max()
