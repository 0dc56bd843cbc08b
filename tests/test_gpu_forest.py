"""Batched forests: independent trees of uneven depth solved in one set of
launches per level (concatenated box lists, per-tree convergence masks),
against per-tree oracle solves."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import rel_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_forest(n, box_n=8, cap=7, seed0=1000):
    params = W.forest2d_params(n, seed0)
    oracles, trees, rhos, bs = [], [], [], []
    for prm in params:
        prm = dict(prm, max_level=min(prm["max_level"], cap))
        p = W.forest2d_problem(prm, box_n)
        a = OracleTree(2, box_n, p.max_level)
        t = afgpu.Tree(2, box_n, p.max_level)
        p.build(a)
        p.build(t)
        rho, b = p.data(a)
        oracles.append(a); trees.append(t); rhos.append(rho); bs.append(b)
    return oracles, trees, rhos, bs


@pytest.mark.parametrize("precision", [afgpu.AFG_FP64, afgpu.AFG_MIXED])
def test_forest_matches_per_tree_oracle(precision):
    oracles, trees, rhos, bs = make_forest(12)
    f = afgpu.Forest(trees)
    assert list(f.cells) == [a.n_leaf_cells for a in oracles]
    f.set_rhs(torch.tensor(np.concatenate(rhos), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate(bs), device="cuda"))
    # the mixed solve is taken to 1e-11: some trees' FP64 round-off floor of
    # the relative residual (cancellation in rho - A u) lies near 1e-12
    tol = 1e-10 if precision == afgpu.AFG_FP64 else 1e-11
    st = f.solve(afgpu.default_opts(rel_tol=tol, precision=precision, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off = 0
    for k, a in enumerate(oracles):
        a.set_rhs(rhos[k]); a.set_dirichlet(bs[k]); a.zero_solution()
        ca = a.solve(tol if precision == afgpu.AFG_FP64 else 1e-12, 60)
        n = a.n_leaf_cells
        assert st[k]["rel_residual"] <= tol
        if precision == afgpu.AFG_FP64:
            assert st[k]["cycles"] == ca  # masked trees stop exactly when they converge
            assert rel_diff(u[off:off + n], a.get_solution()) <= 1e-12
        else:
            assert rel_diff(u[off:off + n], a.get_solution()) <= 1e-8
        off += n


def test_forest_with_one_tree_equals_tree_solve():
    oracles, trees, rhos, bs = make_forest(1)
    f = afgpu.Forest(trees)
    f.set_rhs(torch.tensor(rhos[0], device="cuda"))
    f.set_dirichlet(torch.tensor(bs[0], device="cuda"))
    f.solve(afgpu.default_opts(rel_tol=1e-10))
    t = trees[0]
    t.set_rhs(torch.tensor(rhos[0], device="cuda"))
    t.set_dirichlet(torch.tensor(bs[0], device="cuda"))
    t.set_solution(torch.zeros(len(rhos[0]), dtype=torch.float64, device="cuda"))
    t.solve(afgpu.default_opts(rel_tol=1e-10))
    assert torch.equal(f.get_solution(), t.get_solution())
