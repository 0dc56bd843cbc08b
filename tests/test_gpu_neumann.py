"""Neumann domain sides on the GPU (CUDA kernels through the C ABI) against
the FP64 CPU oracle on the same seeded inputs: cycle-by-cycle FP64 parity
(1e-12 relative max-norm after the same cycles), mixed precision (1e-8),
the adjoint (transposed operator and dL/db on Neumann faces), and forests
whose trees have different side types.  Sec. 2 and 3 of arXiv:1701.04329
allow Dirichlet, Neumann or a mix; b on a Neumann side is the outward normal
derivative and the ghost u + h b."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import load, pair_random, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TYPES = {2: [[1, 0, 0, 1], [0, 0, 1, 1], [1, 1, 0, 1]],
         3: [[1, 0, 1, 0, 0, 1], [0, 1, 1, 1, 1, 1], [1, 1, 0, 0, 1, 1]]}


def neumann_pair(D, N, uni, extra, seed, types):
    a, b, rho, bv = pair_random(D, N, uni, extra, seed)
    a.set_boundary_types(types)
    b.set_boundary_types(types)
    return a, b, rho, bv


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 3, 71), (2, 8, 1, 3, 72), (2, 16, 1, 2, 73),
                                               (3, 4, 1, 3, 74), (3, 8, 2, 2, 75), (3, 16, 1, 1, 76)])
def test_neumann_cycle_by_cycle(D, N, uni, extra, seed):
    for types in TYPES[D]:
        a, b, rho, bv = neumann_pair(D, N, uni, extra, seed, types)
        load(a, b, rho, bv)
        cycles_parity(a, b, 2)


@pytest.mark.parametrize("D,N", [(2, 8), (3, 8)])
def test_neumann_single_box_uniform_and_graph_off(D, N):
    """Levels at and below the root box only (the one-launch bottom solve),
    one uniform level above it, and the per-kernel path without graphs."""
    for lvl in (1, 2):
        a, b, rho, bv = neumann_pair(D, N, lvl, 0, 80 + lvl, TYPES[D][0])
        load(a, b, rho, bv)
        cycles_parity(a, b, 2)
    a, b, rho, bv = neumann_pair(D, N, 2, 1, 83, TYPES[D][2])
    load(a, b, rho, bv)
    cycles_parity(a, b, 2, afgpu.default_opts(n_down=1, n_up=3, n_base=6, use_graph=0))


@pytest.mark.parametrize("D", [2, 3])
def test_neumann_solve_and_mixed_precision(D):
    """Solve to tolerance: same cycle count as the oracle (FP64); the
    FP32 + FP64 defect correction reaches the FP64 tolerance and the
    oracle's solution within 1e-8."""
    a, b, rho, bv = neumann_pair(D, 8, 2 if D == 2 else 1, 2, 90 + D, TYPES[D][1])
    load(a, b, rho, bv)
    ca = a.solve(1e-10, 60)
    sb = b.solve(afgpu.default_opts(rel_tol=1e-10))
    assert sb["cycles"] == ca
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
    a.zero_solution()
    a.solve(1e-12, 60)
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    sb = b.solve(afgpu.default_opts(rel_tol=1e-11, precision=afgpu.AFG_MIXED, max_cycles=60))
    assert sb["rel_residual"] <= 1e-11
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 2, 95), (3, 8, 1, 2, 96)])
def test_neumann_adjoint_matches_transpose_solve(D, N, uni, extra, seed):
    a, b, rho, bv = neumann_pair(D, N, uni, extra, seed, TYPES[D][0])
    g = np.random.default_rng(seed).normal(size=a.n_leaf_cells)
    ref = oadj.direct(a, g)
    lam, db, st = b.adjoint(torch.tensor(g, device="cuda"), afgpu.default_opts(rel_tol=1e-12, max_cycles=100))
    assert st["rel_residual"] <= 1e-12
    lam = lam.cpu().numpy()
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()
    dref = oadj.dl_db(a, ref)
    assert np.abs(db.cpu().numpy() - dref).max() <= 1e-9 * np.abs(dref).max()


def test_neumann_forest_matches_per_tree_oracle():
    """Trees with different side types in one forest (each keeps its own)."""
    params = W.forest2d_params(6, 2000)
    oracles, trees, rhos, bs = [], [], [], []
    for k, prm in enumerate(params):
        prm = dict(prm, max_level=min(prm["max_level"], 6))
        p = W.forest2d_problem(prm, 8)
        a = OracleTree(2, 8, p.max_level)
        t = afgpu.Tree(2, 8, p.max_level)
        p.build(a)
        p.build(t)
        types = TYPES[2][k % 3] if k % 2 else [0, 0, 0, 0]
        a.set_boundary_types(types)
        t.set_boundary_types(types)
        rho, b = p.data(a)
        oracles.append(a); trees.append(t); rhos.append(rho); bs.append(b)
    f = afgpu.Forest(trees)
    f.set_rhs(torch.tensor(np.concatenate(rhos), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate(bs), device="cuda"))
    st = f.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off = 0
    for k, a in enumerate(oracles):
        a.set_rhs(rhos[k]); a.set_dirichlet(bs[k]); a.zero_solution()
        ca = a.solve(1e-10, 60)
        n = a.n_leaf_cells
        assert st[k]["cycles"] == ca
        assert rel_diff(u[off:off + n], a.get_solution()) <= TOL64
        off += n
