"""Periodic domain sides on the GPU (CUDA kernels through the C ABI) against
the FP64 CPU oracle on the same seeded inputs: cycle-by-cycle FP64 parity
(1e-12 relative after the same cycles), solves and mixed precision, the
adjoint, forests.  Sec. 2.2 of arXiv:1701.04329 imposes periodicity through
the connectivity (the box beyond the last one is the first); below the root
each level has one box, its own neighbour across a periodic side."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import load, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TYPES = {2: [[2, 2, 0, 0], [2, 2, 1, 0], [0, 1, 2, 2]],
         3: [[2, 2, 0, 0, 2, 2], [0, 1, 2, 2, 0, 0], [2, 2, 2, 2, 0, 1]]}


def periodic_pair(D, N, uniform, extra, seed, types, frac=0.35, n_buf=1):
    rng = np.random.default_rng(seed)
    a = OracleTree(D, N, uniform + extra)
    b = afgpu.Tree(D, N, uniform + extra)
    for t in (a, b):
        t.set_boundary_types(types)
        t.refine_uniform(uniform)
    for _ in range(extra):
        flags = np.repeat((rng.random(a.nleaf) < frac).astype(np.int8), N ** D)
        a.adapt(flags, n_buf)
        b.adapt(flags, n_buf)
    x = a.cell_centers()
    rho = np.sin(2 * np.pi * x[:, 0] + 1) * np.cos(2 * np.pi * x[:, 1]) + rng.normal(scale=0.1, size=len(x))
    bv = rng.normal(size=a.n_bfaces)
    return a, b, rho, bv


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 3, 121), (2, 8, 1, 3, 122), (2, 16, 1, 2, 123),
                                               (3, 4, 1, 3, 124), (3, 8, 2, 2, 125), (3, 16, 1, 1, 126)])
def test_periodic_cycle_by_cycle(D, N, uni, extra, seed):
    for types in TYPES[D]:
        a, b, rho, bv = periodic_pair(D, N, uni, extra, seed, types)
        load(a, b, rho, bv)
        cycles_parity(a, b, 2)


@pytest.mark.parametrize("D,N", [(2, 8), (3, 8)])
def test_periodic_root_box_uniform_and_graph_off(D, N):
    """The root box alone (its own neighbour across the periodic sides, all
    levels in the one-launch bottom solve), one uniform level, and the
    per-kernel path without graphs."""
    for lvl in (1, 2):
        a, b, rho, bv = periodic_pair(D, N, lvl, 0, 130 + lvl, TYPES[D][0])
        load(a, b, rho, bv)
        cycles_parity(a, b, 2)
    a, b, rho, bv = periodic_pair(D, N, 2, 1, 133, TYPES[D][1])
    load(a, b, rho, bv)
    cycles_parity(a, b, 2, afgpu.default_opts(n_down=1, n_up=3, n_base=6, use_graph=0))


@pytest.mark.parametrize("D", [2, 3])
def test_periodic_solve_and_mixed_precision(D):
    a, b, rho, bv = periodic_pair(D, 8, 2 if D == 2 else 1, 2, 140 + D, TYPES[D][0])
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


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 2, 145), (3, 8, 1, 2, 146)])
def test_periodic_adjoint_matches_transpose_solve(D, N, uni, extra, seed):
    a, b, rho, bv = periodic_pair(D, N, uni, extra, seed, TYPES[D][1])
    g = np.random.default_rng(seed).normal(size=a.n_leaf_cells)
    ref = oadj.direct(a, g)
    lam, db, st = b.adjoint(torch.tensor(g, device="cuda"), afgpu.default_opts(rel_tol=1e-12, max_cycles=100))
    assert st["rel_residual"] <= 1e-12
    lam = lam.cpu().numpy()
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()
    dref = oadj.dl_db(a, ref)
    assert np.abs(db.cpu().numpy() - dref).max() <= 1e-9 * np.abs(dref).max()


def test_periodic_forest_matches_per_tree_oracle():
    """Periodic and non-periodic trees of uneven depth in one forest."""
    params = W.forest2d_params(6, 3000)
    oracles, trees, rhos, bs = [], [], [], []
    for k, prm in enumerate(params):
        prm = dict(prm, max_level=min(prm["max_level"], 6))
        p = W.forest2d_problem(prm, 8)
        types = TYPES[2][k % 3] if k % 2 else [0, 0, 0, 0]
        a = OracleTree(2, 8, p.max_level)
        t = afgpu.Tree(2, 8, p.max_level)
        for x in (a, t):
            x.set_boundary_types(types)
            p.build(x)
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
