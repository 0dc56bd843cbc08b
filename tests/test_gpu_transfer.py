"""Mesh adaptation with the solution carried along, on the GPU (arXiv:
1701.04329 Sec. 2.3 and 2.5; afg_adapt_transfer) against the oracle's
ot_adapt_transfer on the same seeded trees, fields and flags: kept leaves
bit for bit, derefined boxes (means of their children) and prolonged new
children (linear, bi/trilinear with edge/corner ghosts, zeroth order) within
1e-14 relative, over random sequences of refinement and derefinement, with
Dirichlet, Neumann and periodic sides."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from tests.gpu_helpers import rel_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def field(x):
    return np.sin(3 * x[:, 0] + 0.5) * np.cos(2 * x[:, 1]) + x[:, 0] ** 2 + (x[:, -1] if x.shape[1] == 3 else 0.0)


@pytest.mark.parametrize("D,N,types", [(2, 8, None), (2, 4, [1, 0, 2, 2]), (2, 16, [0, 1, 0, 0]),
                                       (3, 4, None), (3, 8, [2, 2, 0, 1, 0, 0])])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_adapt_transfer_matches_the_oracle(D, N, types, scheme):
    rng = np.random.default_rng(900 + 10 * D + N + scheme)
    a, b = OracleTree(D, N, 5), afgpu.Tree(D, N, 5)
    for t in (a, b):
        if types is not None:
            t.set_boundary_types(types)
        t.refine_uniform(2)
    for step in range(4):
        x = a.cell_centers()
        u = field(x) + 0.01 * rng.normal(size=len(x))
        bv = rng.normal(size=a.n_bfaces)
        a.set_dirichlet(bv)
        b.set_dirichlet(torch.tensor(bv, device="cuda"))
        b.set_solution(torch.tensor(u, device="cuda"))
        # per leaf box: refine, derefine or keep (derefinement needs all siblings flagged)
        choice = rng.choice([1, -1, 0], size=a.nleaf, p=[0.25, 0.45, 0.30])
        flags = np.repeat(choice.astype(np.int8), N ** D)
        un, added, removed = a.adapt_transfer(flags, u, 1, scheme)
        added_b, removed_b = b.adapt_transfer(flags, 1, scheme)
        assert (added_b, removed_b) == (added, removed)
        ub = b.get_solution().cpu().numpy()
        assert ub.shape == un.shape
        assert rel_diff(ub, un) <= 1e-14, (step, rel_diff(ub, un))
    assert a.nleaf == b.info().n_leaves


def test_transfer_then_solve():
    """After the transfer the tree is ready for new data and a solve, warm
    started from the carried solution."""
    a, b = OracleTree(2, 8, 5), afgpu.Tree(2, 8, 5)
    for t in (a, b):
        t.refine_uniform(3)
    x = a.cell_centers()
    rho = np.exp(-((x - 0.5) ** 2).sum(1) / 0.01)
    b.set_rhs(torch.tensor(rho, device="cuda"))
    b.solve(afgpu.default_opts(rel_tol=1e-10))
    flags = (np.abs(rho) > 0.1).astype(np.int8)
    b.adapt_transfer(flags, 2, 1)
    a.adapt(flags, 2)
    x = a.cell_centers()
    rho = np.exp(-((x - 0.5) ** 2).sum(1) / 0.01)
    b.set_rhs(torch.tensor(rho, device="cuda"))
    st = b.solve(afgpu.default_opts(rel_tol=1e-10))
    a.set_rhs(rho); a.set_dirichlet(np.zeros(a.n_bfaces)); a.zero_solution()
    a.solve(1e-12, 60)
    assert st["rel_residual"] <= 1e-10
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8


def test_transfer_needs_device_data():
    t = afgpu.Tree(2, 8, 3)
    t.refine_uniform(2)
    with pytest.raises(afgpu.AfgError) as e:
        t.adapt_transfer(np.zeros(t.n_leaf_cells, np.int8))
    assert e.value.code == afgpu.AFG_ERR_STATE


def test_device_flags_equal_the_criterion():
    """afg_flag_cells against the same criterion evaluated in numpy on the
    oracle's cell sizes (the decisions are integers: equal everywhere)."""
    from paper_1701_04329_gb300 import workloads as W
    p = W.gauss2d(max_level=6)
    a, b = OracleTree(2, 8, 6), afgpu.Tree(2, 8, 6)
    p.build(a)
    p.build(b)
    x = a.cell_centers()
    f = p.rho(x)
    h, _ = W.leaf_cell_h(a)
    for power, tr, tc in ((2, 1e-4, 1e-7), (0, 50.0, 1.0), (1, 1e-2, -1.0)):
        hp = np.ones_like(h)
        for _ in range(power):
            hp = hp * h
        v = np.abs(f) * hp
        want = np.where(v > tr, 1, np.where(v < tc, -1, 0)).astype(np.int8)
        got = b.flag_cells(torch.tensor(f, device="cuda"), power, tr, tc).cpu().numpy()
        assert np.array_equal(got, want)


def test_adaptation_loop_on_the_device_builds_the_oracle_tree():
    """The refinement loop of the 2D Gaussian workload driven by device
    flags and afg_adapt_transfer gives the tree the oracle builds with the
    host criterion (bit-exact tree arrays)."""
    from paper_1701_04329_gb300 import workloads as W
    p = W.gauss2d(max_level=6)
    a = OracleTree(2, 8, 6)
    p.build(a)
    b = afgpu.Tree(2, 8, 6)
    b.refine_uniform(p.uniform_level)
    for _ in range(10):
        x = b.cell_centers()
        b.set_solution(torch.zeros(len(x), dtype=torch.float64, device="cuda"))
        fl = b.flag_cells(torch.tensor(p.rho(x), device="cuda"), 2, 1e-4, -1.0).cpu().numpy()
        h, lv = W.leaf_cell_h(b)
        fl[lv >= 6] = np.minimum(fl[lv >= 6], 0)
        if not (fl > 0).any():
            break
        added, removed = b.adapt_transfer(fl, 2, 0)
        if added == 0 and removed == 0:
            break
    ea, eb = a.export(), b.export()
    for k in ("level", "idx", "parent", "children", "neighbours"):
        assert np.array_equal(ea[k], eb[k]), k
