"""Variable-coefficient operators on the GPU (arXiv:1701.04329 Sec. 3.4:
div(eps grad u) with harmonic-mean face coefficients; Sec. 3.5: the same in
(r,z) coordinates with volume-weighted restriction) against the FP64 CPU
oracle on the same seeded inputs: cycle by cycle at 1e-12 (relative
max-norm, after the same cycles), solves to a tolerance with the oracle's
cycle count, mixed precision within 1e-8 of the oracle's converged FP64
solution, and the paper's jump layout (eps = 100 on [0,1/4]^2)."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from tests.gpu_helpers import load, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def var_pair(D, N, uniform, extra, seed, op, types=None, frac=0.3, lo=0.1, hi=100.0, cells=None):
    """The same random AMR tree on both sides, eps log-uniform in [lo, hi]
    and constant on each of cells^D blocks of the domain (default N: the
    level-1 cells), a smooth source with noise, random boundary data.
    cells = 2 puts the jumps on faces of the coarsest (2^D-cell) grid, as
    Sec. 3.4 asks for fast convergence."""
    cells = N if cells is None else cells
    rng = np.random.default_rng(seed)
    a = OracleTree(D, N, uniform + extra)
    b = afgpu.Tree(D, N, uniform + extra)
    for t in (a, b):
        if types is not None:
            t.set_boundary_types(types)
        t.refine_uniform(uniform)
    for _ in range(extra):
        flags = np.repeat((rng.random(a.nleaf) < frac).astype(np.int8), N ** D)
        a.adapt(flags, 1)
        b.adapt(flags, 1)
    x = a.cell_centers()
    table = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(cells,) * D))
    eps = table[tuple(np.minimum((x[:, k] * cells).astype(int), cells - 1) for k in range(D))]
    rho = np.sin(5 * x[:, 0] + 1) * np.cos(3 * x[:, 1]) + rng.normal(scale=0.1, size=len(x))
    bv = rng.normal(size=a.n_bfaces)
    a.set_operator(op)
    b.set_operator(op)
    a.set_eps(eps)
    b.set_eps(torch.tensor(eps, device="cuda"))
    return a, b, rho, bv, eps


@pytest.mark.parametrize("D,N,uni,extra,op,seed", [
    (2, 8, 2, 2, 1, 701), (2, 4, 2, 3, 1, 702), (2, 16, 1, 2, 1, 703), (3, 8, 1, 2, 1, 704), (3, 4, 2, 2, 1, 705),
    (2, 8, 2, 2, 2, 706), (2, 4, 2, 3, 2, 707), (2, 16, 1, 2, 2, 708)])
def test_var_cycle_by_cycle(D, N, uni, extra, op, seed):
    a, b, rho, bv, _ = var_pair(D, N, uni, extra, seed, op)
    load(a, b, rho, bv)
    cycles_parity(a, b, 3)


@pytest.mark.parametrize("types,op", [([1, 0, 0, 0], 1), ([0, 0, 2, 2], 1), ([1, 0, 0, 1], 2)])
def test_var_other_sides_cycle_by_cycle(types, op):
    a, b, rho, bv, _ = var_pair(2, 8, 2, 2, 710 + op, op, types=types)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("op", [1, 2])
def test_var_solve_and_mixed(op):
    # jumps on the coarsest grid's faces, a moderate range: the FP64 round-off floor of the
    # relative residual (about 4e-11 here with random boundary data) stays below the tolerance
    a, b, rho, bv, _ = var_pair(2, 8, 2, 3, 720 + op, op, cells=2, lo=0.5, hi=4.0)
    load(a, b, rho, bv)
    ca = a.solve(1e-10, 60)
    assert ca < 60
    st = b.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=60))
    assert st["cycles"] == ca
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
    a.solve(1e-12, 80)  # on to the round-off floor
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    sm = b.solve(afgpu.default_opts(rel_tol=1e-10, precision=afgpu.AFG_MIXED, max_cycles=60))
    assert sm["rel_residual"] <= 1e-10
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8


@pytest.mark.parametrize("op", [1, 2])
def test_paper_jump_layout(op):
    """Sec. 4.1's second test: eps = 100 on [0,1/4]^2, 1 elsewhere, two
    Gaussian sources at (1/4,1/4) and (3/4,3/4), u = 0 on the sides; 128^2
    cells plus one refinement level around the sources."""
    a = OracleTree(2, 8, 6)
    b = afgpu.Tree(2, 8, 6)
    for t in (a, b):
        t.refine_uniform(5)
    x = a.cell_centers()
    src = lambda p: sum(np.exp(-np.sum((p - c) ** 2, 1) / 0.04 ** 2) for c in ((0.25, 0.25), (0.75, 0.75)))
    flags = (np.abs(src(x)) > 0.05).astype(np.int8)
    a.adapt(flags, 2)
    b.adapt(flags, 2)
    x = a.cell_centers()
    eps = np.where((x[:, 0] < 0.25) & (x[:, 1] < 0.25), 100.0, 1.0)
    rho = src(x)
    for t in (a, b):
        t.set_operator(op)
    a.set_eps(eps)
    b.set_eps(torch.tensor(eps, device="cuda"))
    load(a, b, rho, np.zeros(a.n_bfaces))
    cycles_parity(a, b, 2)
    a.zero_solution()
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    ca = a.solve(1e-10, 60)
    st = b.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=60))
    assert st["cycles"] == ca
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64


def test_var_forest_matches_per_tree_oracle():
    pairs = [var_pair(2, 8, 2, 2, 730 + k, 1, cells=2, lo=0.5, hi=4.0) for k in range(4)]
    f = afgpu.Forest([p[1] for p in pairs])
    f.set_eps(torch.tensor(np.concatenate([p[4] for p in pairs]), device="cuda"))
    f.set_rhs(torch.tensor(np.concatenate([p[2] for p in pairs]), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate([p[3] for p in pairs]), device="cuda"))
    st = f.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off = 0
    for k, (a, _, rho, bv, _) in enumerate(pairs):
        a.set_rhs(rho); a.set_dirichlet(bv); a.zero_solution()
        ca = a.solve(1e-10, 60)
        n = a.n_leaf_cells
        assert st[k]["cycles"] == ca
        assert rel_diff(u[off:off + n], a.get_solution()) <= TOL64
        off += n


def test_var_calls_need_eps_and_refuse_what_is_not_built():
    t = afgpu.Tree(2, 8, 3)
    t.refine_uniform(2)
    n = t.n_leaf_cells
    t.set_rhs(torch.ones(n, dtype=torch.float64, device="cuda"))
    t.set_operator(afgpu.AFG_OP_VAR)
    with pytest.raises(afgpu.AfgError) as e:
        t.solve()
    assert e.value.code == afgpu.AFG_ERR_STATE and "eps" in str(e.value)
    t.set_eps(torch.ones(n, dtype=torch.float64, device="cuda"))
    t.solve(afgpu.default_opts(rel_tol=1e-8))
    with pytest.raises(afgpu.AfgError) as e:
        t.adjoint(torch.ones(n, dtype=torch.float64, device="cuda"))
    assert e.value.code == afgpu.AFG_ERR_STATE
    with pytest.raises(afgpu.AfgError):
        afgpu.Tree(3, 8, 2).set_operator(afgpu.AFG_OP_VAR_RZ)
