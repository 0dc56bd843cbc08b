"""The bi/trilinear and zeroth-order prolongations of the coarse-grid
correction on the GPU (arXiv:1701.04329 Sec. 2.5, with the edge/corner
ghosts of Sec. 2.4 for the bi/trilinear scheme) against the FP64 CPU oracle
(ot_set_prolong) on the same seeded inputs: cycle by cycle at 1e-12
(relative max-norm, after the same cycles), with Neumann and periodic sides
(diagonal neighbours across a periodic side), with the variable-coefficient
operator, and a solve to a tolerance with the oracle's cycle count."""
import numpy as np
import pytest

from paper_1701_04329_gb300 import afgpu
from tests.gpu_helpers import load, pair_random, rel_diff
from tests.test_gpu_parity import TOL64, cycles_parity
from tests.test_gpu_varcoef import var_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def with_scheme(a, b, scheme):
    a.set_prolong(scheme)
    b.set_prolongation(scheme)


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 8, 2, 2, 801), (2, 4, 2, 3, 802), (2, 16, 1, 2, 803),
                                               (3, 8, 1, 2, 804), (3, 4, 2, 2, 805)])
@pytest.mark.parametrize("scheme", [afgpu.AFG_PROLONG_MULTILINEAR, afgpu.AFG_PROLONG_ZEROTH])
def test_prolongation_cycle_by_cycle(D, N, uni, extra, seed, scheme):
    a, b, rho, bv = pair_random(D, N, uni, extra, seed)
    with_scheme(a, b, scheme)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("D,types", [(2, [1, 0, 0, 1]), (2, [2, 2, 0, 0]), (2, [2, 2, 1, 0]),
                                     (3, [2, 2, 2, 2, 0, 0]), (3, [1, 0, 2, 2, 0, 1])])
def test_multilinear_with_other_sides(D, types):
    rng = np.random.default_rng(810 + D)
    from oracle.oracle import OracleTree
    N = 8 if D == 2 else 4
    a, b = OracleTree(D, N, 4), afgpu.Tree(D, N, 4)
    for t in (a, b):
        t.set_boundary_types(types)
        t.refine_uniform(2)
    for _ in range(2):
        flags = np.repeat((rng.random(a.nleaf) < 0.3).astype(np.int8), N ** D)
        a.adapt(flags, 1)
        b.adapt(flags, 1)
    x = a.cell_centers()
    rho = np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]) + rng.normal(scale=0.1, size=len(x))
    bv = rng.normal(size=a.n_bfaces)
    with_scheme(a, b, afgpu.AFG_PROLONG_MULTILINEAR)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("op", [1, 2])
def test_multilinear_with_variable_coefficients(op):
    a, b, rho, bv, _ = var_pair(2, 8, 2, 2, 820 + op, op)
    with_scheme(a, b, afgpu.AFG_PROLONG_MULTILINEAR)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("scheme", [afgpu.AFG_PROLONG_MULTILINEAR, afgpu.AFG_PROLONG_ZEROTH])
def test_prolongation_solve_and_mixed(scheme):
    a, b, rho, bv = pair_random(2, 8, 2, 3, 830 + scheme)
    with_scheme(a, b, scheme)
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
