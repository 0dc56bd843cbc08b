"""Batched forests: independent trees of uneven depth solved in one set of
launches per level (concatenated box lists, per-tree convergence masks),
against per-tree oracle solves.

The full batched workload is tested at its own size: 512 quadtrees (seeds
1000 + t, 1-4 Gaussian sources, maximum level drawn from 4..9, so box counts
differ about 100-fold), with boxes of 8^2 and of 16^2 cells.  FP64: every
tree stops after the oracle's number of cycles and matches the oracle's
solution after those cycles within 1e-12 (relative max-norm).  Mixed
precision: every tree reaches the FP64 tolerance and is within 1e-8 of the
oracle's converged FP64 solution."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import rel_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_TREES = 512
TOL = 1e-10


def make_forest(n, box_n=8, cap=None, seed0=1000):
    params = W.forest2d_params(n, seed0)
    oracles, trees, rhos, bs = [], [], [], []
    for prm in params:
        if cap is not None:
            prm = dict(prm, max_level=min(prm["max_level"], cap))
        p = W.forest2d_problem(prm, box_n)
        a = OracleTree(2, box_n, p.max_level)
        t = afgpu.Tree(2, box_n, p.max_level)
        p.build(a)
        p.build(t)
        rho, b = p.data(a)
        oracles.append(a); trees.append(t); rhos.append(rho); bs.append(b)
    return oracles, trees, rhos, bs


@pytest.fixture(scope="module", params=[8, 16], ids=["box8", "box16"])
def c3(request):
    """The batched workload built on the oracle and the library, and the
    oracle's per-tree results: cycles and solution at TOL, and the solution
    taken on to the FP64 floor (rel. residual 1e-12, or 12 more cycles)."""
    box_n = request.param
    trees, rhos, bs, cells, cycles, u_tol, u_conv = [], [], [], [], [], [], []
    for prm in W.forest2d_params(N_TREES, 1000):
        p = W.forest2d_problem(prm, box_n)
        a = OracleTree(2, box_n, p.max_level)
        t = afgpu.Tree(2, box_n, p.max_level)
        p.build(a)
        p.build(t)
        rho, b = p.data(a)
        a.set_rhs(rho); a.set_dirichlet(b); a.zero_solution()
        cycles.append(a.solve(TOL, 60))
        u_tol.append(a.get_solution())
        for _ in range(12):
            r, pm = a.residual_norm()
            if r <= 1e-12 * pm:
                break
            a.vcycle()
        u_conv.append(a.get_solution())
        cells.append(a.n_leaf_cells)
        trees.append(t); rhos.append(rho); bs.append(b)
        del a
    f = afgpu.Forest(trees)
    assert list(f.cells) == cells
    levels = [t.info().highest_level for t in trees]
    return dict(box_n=box_n, forest=f, rho=np.concatenate(rhos), b=np.concatenate(bs), cells=cells,
                cycles=cycles, u_tol=u_tol, u_conv=u_conv, levels=levels)


def _load(c):
    f = c["forest"]
    f.set_rhs(torch.tensor(c["rho"], device="cuda"))
    f.set_dirichlet(torch.tensor(c["b"], device="cuda"))
    return f


def test_c3_workload_shape(c3):
    """The workload spans what it should: 512 trees, finest levels 4..9 (one
    fewer with 16^2 boxes), leaf counts differing by far more than 10x."""
    shift = 0 if c3["box_n"] == 8 else 1
    assert len(c3["cells"]) == N_TREES
    assert min(c3["levels"]) <= 5 - shift and max(c3["levels"]) == 9 - shift
    assert max(c3["cells"]) / min(c3["cells"]) > 100


def test_c3_fp64_matches_oracle_cycle_for_cycle(c3):
    f = _load(c3)
    st = f.solve(afgpu.default_opts(rel_tol=TOL, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off, worst = 0, 0.0
    for k, n in enumerate(c3["cells"]):
        assert st[k]["rel_residual"] <= TOL, k
        assert st[k]["cycles"] == c3["cycles"][k], (k, st[k]["cycles"], c3["cycles"][k])
        worst = max(worst, rel_diff(u[off:off + n], c3["u_tol"][k]))
        off += n
    assert worst <= 1e-12, worst


def test_c3_mixed_within_1e8_of_the_fp64_oracle(c3):
    f = _load(c3)
    st = f.solve(afgpu.default_opts(rel_tol=TOL, precision=afgpu.AFG_MIXED, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off, worst = 0, 0.0
    for k, n in enumerate(c3["cells"]):
        assert st[k]["rel_residual"] <= TOL, k
        worst = max(worst, rel_diff(u[off:off + n], c3["u_conv"][k]))
        off += n
    assert worst <= 1e-8, worst


@pytest.mark.parametrize("precision", [afgpu.AFG_FP64, afgpu.AFG_MIXED])
def test_small_forest_matches_per_tree_oracle(precision):
    oracles, trees, rhos, bs = make_forest(12, cap=7)
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
    oracles, trees, rhos, bs = make_forest(1, cap=7)
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
