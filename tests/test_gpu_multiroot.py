"""Trees whose level 1 is a block of root boxes on the GPU (the one-CTA block
bottom solve, or -- beyond one CTA's shared memory and in forests -- their
coarse grids as device boxes on the per-level kernels; CUDA kernels through
the C ABI) against the FP64 CPU oracle on the same seeded inputs:
cycle-by-cycle FP64 parity (1e-12 relative after the same cycles), solves
and mixed precision.  Sec. 2.2 of arXiv:1701.04329
(several root boxes) and Sec. 3.2 (several boxes on the coarse grids)."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu
from tests.gpu_helpers import load, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def block_pair(D, N, roots, uniform, extra, seed, types=None, frac=0.35, n_buf=1):
    rng = np.random.default_rng(seed)
    a = OracleTree(D, N, uniform + extra, roots=roots)
    b = afgpu.Tree(D, N, uniform + extra, roots=roots)
    for t in (a, b):
        if types is not None:
            t.set_boundary_types(types)
        t.refine_uniform(uniform)
    for _ in range(extra):
        flags = np.repeat((rng.random(a.nleaf) < frac).astype(np.int8), N ** D)
        a.adapt(flags, n_buf)
        b.adapt(flags, n_buf)
    x = a.cell_centers()
    rho = np.sin(3 * x[:, 0] + 1) * np.cos(2 * x[:, 1]) + rng.normal(scale=0.1, size=len(x))
    bv = rng.normal(size=a.n_bfaces)
    return a, b, rho, bv


@pytest.mark.parametrize("D,N,roots,uni,extra,types,seed", [
    (2, 8, (2, 1), 1, 2, None, 601), (2, 8, (3, 2), 1, 2, [0, 1, 0, 0], 602),
    (2, 4, (1, 3), 2, 2, [2, 2, 0, 0], 603), (2, 16, (2, 1), 1, 1, [0, 0, 2, 2], 604),
    (3, 8, (2, 1, 1), 1, 1, None, 605), (3, 4, (1, 2, 2), 1, 2, [0, 1, 2, 2, 0, 0], 606)])
def test_block_cycle_by_cycle(D, N, roots, uni, extra, types, seed):
    a, b, rho, bv = block_pair(D, N, roots, uni, extra, seed, types)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("D,roots", [(2, (3, 1)), (3, (2, 1, 1))])
def test_roots_only_and_graph_off(D, roots):
    """The tree is its root boxes alone (the whole cycle in the block bottom
    solve), and the per-kernel path without graphs."""
    a, b, rho, bv = block_pair(D, 8, roots, 1, 0, 610 + D)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)
    a, b, rho, bv = block_pair(D, 8, roots, 1, 1, 612 + D)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2, afgpu.default_opts(n_down=1, n_up=3, n_base=6, use_graph=0))


@pytest.mark.parametrize("D", [2, 3])
def test_block_solve_and_mixed_precision(D):
    a, b, rho, bv = block_pair(D, 8, (2, 1) if D == 2 else (2, 1, 1), 2 if D == 2 else 1, 2, 620 + D)
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


@pytest.mark.parametrize("D,roots,op,scheme,seed", [
    (2, (2, 1), afgpu.AFG_OP_VAR, 0, 640), (2, (3, 2), afgpu.AFG_OP_VAR_RZ, 0, 641),
    (2, (1, 3), 0, afgpu.AFG_PROLONG_MULTILINEAR, 642), (3, (2, 1, 1), afgpu.AFG_OP_VAR, 0, 643),
    (3, (1, 2, 1), 0, afgpu.AFG_PROLONG_ZEROTH, 644), (2, (2, 2), afgpu.AFG_OP_VAR, afgpu.AFG_PROLONG_MULTILINEAR, 645)])
def test_block_trees_with_other_operators_cycle_by_cycle(D, roots, op, scheme, seed):
    """A block tree given a variable-coefficient operator (eps log-uniform in
    [0.5, 4] per level-1 cell) or another prolongation before its data keeps
    its coarse grids as device boxes on the per-level kernels; cycle by cycle
    against the oracle."""
    a, b, rho, bv = block_pair(D, 8, roots, 1, 2, seed)
    for t in (a, b):
        if op:
            t.set_operator(op)
        if scheme:
            (t.set_prolong if t is a else t.set_prolongation)(scheme)
    if op:
        rng = np.random.default_rng(seed + 1)
        x = a.cell_centers()
        table = np.exp(rng.uniform(np.log(0.5), np.log(4.0), size=tuple(8 * r for r in roots)))
        eps = table[tuple(np.minimum((x[:, k] * 8).astype(int), 8 * roots[k] - 1) for k in range(D))]
        a.set_eps(eps)
        b.set_eps(torch.tensor(eps, device="cuda"))
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


def test_block_trees_refuse_what_is_not_built():
    """Once the data of a block tree are set for the one-CTA block solve, the
    operator and prolongation stay; singular problems take trees of one root
    box."""
    t = afgpu.Tree(2, 8, 3, roots=(2, 1))
    t.refine_uniform(2)
    t.set_rhs(torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda"))
    for call in (lambda: t.set_operator(afgpu.AFG_OP_VAR), lambda: t.set_prolongation(afgpu.AFG_PROLONG_ZEROTH)):
        with pytest.raises(afgpu.AfgError) as e:
            call()
        assert e.value.code == afgpu.AFG_ERR_STATE
    s = afgpu.Tree(2, 8, 3, roots=(2, 1))
    s.set_boundary_types([2, 2, 1, 1])
    s.refine_uniform(2)
    with pytest.raises(afgpu.AfgError) as e:
        s.set_rhs(torch.zeros(s.n_leaf_cells, dtype=torch.float64, device="cuda"))
    assert e.value.code == afgpu.AFG_ERR_STATE


@pytest.mark.parametrize("D,N,roots,uni,extra,types,seed", [
    (3, 8, (2, 2, 2), 1, 1, None, 620), (3, 8, (7, 1, 1), 1, 1, [2, 2, 0, 0, 1, 0], 621),
    (2, 8, (9, 9), 1, 1, None, 622), (3, 16, (2, 1, 1), 1, 1, [0, 0, 1, 0, 0, 0], 623)])
def test_large_blocks_cycle_by_cycle(D, N, roots, uni, extra, types, seed):
    """Blocks beyond one CTA's shared memory (a 2 x 2 x 2 or 7 x 1 x 1 block
    of 8^3 roots, 9 x 9 of 8^2, any block of 16^3): their coarse grids are
    device boxes, one per root and level, on the per-level kernels."""
    a, b, rho, bv = block_pair(D, N, roots, uni, extra, seed, types=types, frac=0.3)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("roots,fits", [((6, 1, 1), True), ((3, 2, 1), True), ((2, 2, 2), False), ((7, 1, 1), False)])
def test_one_cta_block_bottom_and_per_level_blocks_solve(roots, fits):
    """Blocks of 8^3 roots on either side of the one-CTA limit solve to the
    tolerance with the oracle's cycle count."""
    a = OracleTree(3, 8, 1, roots=roots)
    t = afgpu.Tree(3, 8, 1, roots=roots)
    x = a.cell_centers()
    rho = np.sin(x[:, 0]) + np.cos(2 * x[:, 1]) * x[:, 2]
    load(a, t, rho, np.zeros(a.n_bfaces))
    ca = a.solve(1e-8, 60)
    st = t.solve(afgpu.default_opts(rel_tol=1e-8, max_cycles=60))
    assert st["cycles"] == ca
    assert rel_diff(t.get_solution(), a.get_solution()) <= TOL64


def test_forest_of_block_trees_matches_per_tree_oracle():
    """A forest that holds trees of several root boxes (and one of a single
    root) runs every tree's coarse grids on the per-level kernels."""
    specs = [((2, 1), 630), ((1, 1), 631), ((1, 3), 632), ((3, 2), 633)]
    pairs = [block_pair(2, 8, roots, 1, 2, seed) for roots, seed in specs]
    f = afgpu.Forest([p[1] for p in pairs])
    f.set_rhs(torch.tensor(np.concatenate([p[2] for p in pairs]), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate([p[3] for p in pairs]), device="cuda"))
    st = f.solve(afgpu.default_opts(rel_tol=1e-10, max_cycles=60))
    u = f.get_solution().cpu().numpy()
    off = 0
    for k, (a, _, rho, bv) in enumerate(pairs):
        a.set_rhs(rho); a.set_dirichlet(bv); a.zero_solution()
        ca = a.solve(1e-10, 60)
        n = a.n_leaf_cells
        assert st[k]["cycles"] == ca, (k, st[k]["cycles"], ca)
        assert rel_diff(u[off:off + n], a.get_solution()) <= TOL64
        off += n
