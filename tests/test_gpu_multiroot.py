"""Trees whose level 1 is a block of root boxes on the GPU (the block bottom
solve, CUDA kernels through the C ABI) against the FP64 CPU oracle on the
same seeded inputs: cycle-by-cycle FP64 parity (1e-12 relative after the
same cycles), solves and mixed precision.  Sec. 2.2 of arXiv:1701.04329
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


def test_forest_of_root_blocks_is_refused():
    t1 = afgpu.Tree(2, 8, 3, roots=(2, 1))
    t2 = afgpu.Tree(2, 8, 3)
    for t in (t1, t2):
        t.refine_uniform(2)
    with pytest.raises(afgpu.AfgError):
        afgpu.Forest([t1, t2])


@pytest.mark.parametrize("roots,fits", [((6, 1, 1), True), ((3, 2, 1), True), ((2, 2, 2), False), ((7, 1, 1), False)])
def test_block_size_limit_of_the_one_cta_bottom(roots, fits):
    """The documented limit for blocks of 8^3 root boxes (FP64, one CTA's
    shared memory): 6 x 1 x 1 and 3 x 2 x 1 fit, 2 x 2 x 2 and 7 x 1 x 1 are
    refused when the device grid is built (the first field call), before
    any kernel or graph."""
    t = afgpu.Tree(3, 8, 1, roots=roots)
    rho = torch.ones(t.n_leaf_cells, dtype=torch.float64, device="cuda")
    if fits:
        t.set_rhs(rho)
        st = t.solve(afgpu.default_opts(rel_tol=1e-8, max_cycles=40))
        assert st["rel_residual"] <= 1e-8
    else:
        with pytest.raises(afgpu.AfgError) as e:
            t.set_rhs(rho)
        assert e.value.code == afgpu.AFG_ERR_STATE and "too large" in str(e.value)
