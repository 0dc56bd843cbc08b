"""Pins of the oracle's adjoint: the transpose relation, the symmetric
uniform-grid special case, and BiCGStab against the direct solve."""
import numpy as np
import pytest

from oracle import adjoint, composite
from tests.test_oracle_pins import random_amr


@pytest.mark.parametrize("D,seed", [(2, 41), (3, 42)])
def test_composite_operator_not_symmetric_on_amr_but_on_uniform(D, seed):
    """With refinement boundaries K != K^T, but W K (volume weighted) has
    zero row and column sums in the interior coupling (conservation); on a
    uniform tree K = K^T exactly."""
    t = random_amr(D, 4, 2, 1, seed)
    K = t.leaf_rows()
    assert abs(K - K.T).max() > 1e-3 * abs(K).max()
    u = random_amr(D, 4, 2, 0, seed)
    Ku = u.leaf_rows()
    assert abs(Ku - Ku.T).max() == 0.0


@pytest.mark.parametrize("D,seed", [(2, 43), (2, 44), (3, 45)])
def test_bicgstab_adjoint_matches_direct_transpose_solve(D, seed):
    t = random_amr(D, 4, 2, 2, seed)
    g = np.random.default_rng(seed).normal(size=t.n_leaf_cells)
    ref = adjoint.direct(t, g)
    lam, its = adjoint.bicgstab(t, g, tol=1e-12)
    assert its < 40
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()


def test_adjoint_gradient_equals_finite_differences_of_the_definition():
    """L = g . u with u = K^-1 (rho - B b): dL/drho = K^-T g, dL/db = -B^T K^-T g.
    L is linear, so central differences are exact up to round-off."""
    t = random_amr(2, 4, 2, 2, 46)
    e = t.export()
    K, B = composite.assemble(2, 4, e["level"], e["idx"], e["children"])
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(46)
    g = rng.normal(size=t.n_leaf_cells)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    L = lambda r, bb: g @ spla.spsolve(K.tocsc(), r - B @ bb)
    lam = adjoint.direct(t, g)
    db = adjoint.dl_db(t, lam)
    for i in rng.choice(len(rho), 5, replace=False):
        d = np.zeros_like(rho); d[i] = 1e-3
        fd = (L(rho + d, b) - L(rho - d, b)) / 2e-3
        assert abs(fd - lam[i]) <= 1e-8 * (1 + abs(fd))
    for f in rng.choice(len(b), 5, replace=False):
        d = np.zeros_like(b); d[f] = 1e-3
        fd = (L(rho, b + d) - L(rho, b - d)) / 2e-3
        assert abs(fd - db[f]) <= 1e-8 * (1 + abs(fd))
