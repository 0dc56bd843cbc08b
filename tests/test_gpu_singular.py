"""Singular problems on the GPU (only Neumann and periodic sides; arXiv:
1701.04329 Sec. 2-3, Sec. 4.4's mean-source subtraction) against the FP64
CPU oracle on the same seeded inputs: the source made compatible, the
solution kept at zero volume-weighted mean; cycle by cycle at 1e-12
(relative max-norm, after the same cycles), solves with the oracle's cycle
count, mixed precision within 1e-8 of the oracle's converged solution."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from tests.gpu_helpers import load, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def singular_pair(D, N, uniform, extra, seed, types, frac=0.3):
    rng = np.random.default_rng(seed)
    a, b = OracleTree(D, N, uniform + extra), afgpu.Tree(D, N, uniform + extra)
    for t in (a, b):
        t.set_boundary_types(types)
        t.refine_uniform(uniform)
    for _ in range(extra):
        flags = np.repeat((rng.random(a.nleaf) < frac).astype(np.int8), N ** D)
        a.adapt(flags, 1)
        b.adapt(flags, 1)
    x = a.cell_centers()
    rho = np.sin(2 * np.pi * x[:, 0] + 1) * np.cos(2 * np.pi * x[:, 1]) + rng.normal(scale=0.1, size=len(x)) + 2.0
    bv = rng.normal(size=a.n_bfaces)
    return a, b, rho, bv


@pytest.mark.parametrize("D,N,types,seed", [(2, 8, [1, 1, 1, 1], 901), (2, 8, [2, 2, 2, 2], 902),
                                            (2, 4, [2, 2, 1, 1], 903), (3, 8, [1, 1, 1, 1, 1, 1], 904),
                                            (3, 4, [2, 2, 2, 2, 2, 2], 905), (2, 16, [1, 1, 2, 2], 906)])
def test_singular_cycle_by_cycle(D, N, types, seed):
    a, b, rho, bv = singular_pair(D, N, 2 if N < 16 else 1, 2, seed, types)
    load(a, b, rho, bv)
    cycles_parity(a, b, 3)


@pytest.mark.parametrize("types", [[1, 1, 1, 1], [2, 2, 2, 2]])
def test_singular_solve_and_mixed(types):
    a, b, rho, bv = singular_pair(2, 8, 2, 3, 910 + types[0], types)
    load(a, b, rho, bv)
    ca = a.solve(1e-10, 80)
    st = b.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=80))
    assert st["cycles"] == ca
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
    a.solve(1e-12, 100)
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    sm = b.solve(afgpu.default_opts(rel_tol=1e-10, precision=afgpu.AFG_MIXED, max_cycles=80))
    assert sm["rel_residual"] <= 1e-10
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8


@pytest.mark.parametrize("precision", [afgpu.AFG_FP64, afgpu.AFG_MIXED])
def test_forest_of_singular_and_dirichlet_trees(precision):
    """A forest of singular trees (Neumann, periodic, mixed sides) and a
    Dirichlet tree: each singular tree's source is made compatible and its
    solution kept at zero mean on its own, as the oracle does per tree."""
    specs = [([1, 1, 1, 1], 920), ([2, 2, 2, 2], 921), ([2, 2, 1, 1], 922), ([0, 1, 0, 1], 923)]
    pairs = [singular_pair(2, 8, 2, 2, seed, types) for types, seed in specs]
    f = afgpu.Forest([p[1] for p in pairs])
    f.set_rhs(torch.tensor(np.concatenate([p[2] for p in pairs]), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate([p[3] for p in pairs]), device="cuda"))
    st = f.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=80, precision=precision))
    u = f.get_solution().cpu().numpy()
    off = 0
    for k, (a, _, rho, bv) in enumerate(pairs):
        a.set_rhs(rho); a.set_dirichlet(bv); a.zero_solution()
        n = a.n_leaf_cells
        assert st[k]["rel_residual"] <= 1e-10, k
        if precision == afgpu.AFG_FP64:
            ca = a.solve(1e-10, 80)
            assert st[k]["cycles"] == ca, (k, st[k]["cycles"], ca)
            assert rel_diff(u[off:off + n], a.get_solution()) <= TOL64, k
        else:
            a.solve(1e-12, 100)
            assert rel_diff(u[off:off + n], a.get_solution()) <= 1e-8, k
        off += n


def test_singular_trees_are_refused_where_not_built():
    t = afgpu.Tree(2, 8, 3)
    t.set_boundary_types([1, 1, 1, 1])
    t.refine_uniform(2)
    n = t.n_leaf_cells
    with pytest.raises(afgpu.AfgError) as e:
        s = afgpu.Tree(2, 8, 3, roots=(2, 1))
        s.set_boundary_types([1, 1, 1, 1])
        afgpu.Forest([t, s])
    assert e.value.code == afgpu.AFG_ERR_STATE
    t.set_rhs(torch.ones(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(afgpu.AfgError) as e:
        t.adjoint(torch.ones(n, dtype=torch.float64, device="cuda"))
    assert e.value.code == afgpu.AFG_ERR_STATE
