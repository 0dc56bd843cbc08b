"""GPU (CUDA kernels through the C ABI) against the FP64 CPU oracle, element
by element, on the same seeded inputs (arXiv:1701.04329 Sec. 3.2 cycles).

Tolerance: FP64 solutions after the same number of cycles agree to 1e-12
relative max-norm (the kernels may fuse multiply-adds and sum in another
order; multigrid contracts such rounding differences)."""
import numpy as np
import pytest

from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import load, pair_from_problem, pair_random, rel_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def cycles_parity(a, b, n_v=3, opts=None):
    a_opts = {} if opts is None else dict(n_down=opts.n_down, n_up=opts.n_up, n_base=opts.n_base)
    a.fmg(**a_opts)
    sb = b.fmg(opts)
    ra, pa = a.residual_norm()
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
    assert abs(sb["rel_residual"] - ra / pa) <= 1e-9 * ra / pa + 1e-15
    for _ in range(n_v):
        a.vcycle(**a_opts)
        sb = b.vcycle(opts)
        ra, pa = a.residual_norm()
        assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
        assert abs(sb["rel_residual"] - ra / pa) <= 1e-6 * ra / pa + 1e-12


def test_gauss2d_cycle_by_cycle():
    a, b, rho, bv = pair_from_problem(W.gauss2d())
    load(a, b, rho, bv)
    cycles_parity(a, b, 4)


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 3, 1), (2, 8, 1, 3, 2), (2, 16, 1, 2, 3),
                                               (3, 4, 1, 3, 4), (3, 8, 2, 2, 5), (3, 16, 1, 1, 6)])
def test_random_amr_cycle_by_cycle(D, N, uni, extra, seed):
    a, b, rho, bv = pair_random(D, N, uni, extra, seed)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2)


@pytest.mark.parametrize("D,N", [(2, 4), (2, 8), (3, 8), (3, 16)])
def test_single_box_and_uniform(D, N):
    for lvl in (1, 2):
        a, b, rho, bv = pair_random(D, N, lvl, 0, 7 + lvl)
        load(a, b, rho, bv)
        cycles_parity(a, b, 1)


def test_smoothing_options_and_graph_off():
    a, b, rho, bv = pair_random(2, 8, 2, 2, 11)
    load(a, b, rho, bv)
    cycles_parity(a, b, 2, afgpu.default_opts(n_down=1, n_up=3, n_base=6, use_graph=0))


def test_solve_to_tolerance_same_cycles():
    p = W.twosrc3d(uniform_level=4, extra_levels=2, s=0.04)
    a, b, rho, bv = pair_from_problem(p)
    load(a, b, rho, bv)
    hist = []
    ca = a.solve(1e-10, 40, history=hist)
    sb = b.solve(afgpu.default_opts(rel_tol=1e-10))
    assert sb["cycles"] == ca
    assert rel_diff(b.get_solution(), a.get_solution()) <= TOL64
    # the relative residual carries ~1e-13 absolute round-off (cancellation in rho - A u)
    assert np.allclose(sb["history"][: len(hist)], hist, rtol=1e-6, atol=1e-12)


def test_mixed_precision_matches_fp64_oracle():
    """FP32 multigrid inside FP64 defect correction reaches the FP64 residual
    tolerance and the FP64 oracle's solution within 1e-8 relative."""
    p = W.gauss2d()
    a, b, rho, bv = pair_from_problem(p)
    load(a, b, rho, bv)
    a.solve(1e-12, 60)
    sb = b.solve(afgpu.default_opts(rel_tol=1e-12, precision=afgpu.AFG_MIXED))
    assert sb["rel_residual"] <= 1e-12
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8
    # 3D too
    a, b, rho, bv = pair_from_problem(W.twosrc3d(uniform_level=4, extra_levels=2, s=0.04))
    load(a, b, rho, bv)
    a.solve(1e-12, 60)
    sb = b.solve(afgpu.default_opts(rel_tol=1e-12, precision=afgpu.AFG_MIXED))
    assert sb["rel_residual"] <= 1e-12
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8


@pytest.mark.parametrize("inner", [0, 1, 3])
def test_mixed_precision_inner_cycles(inner):
    """A fixed number of FP32 V-cycles per FP64 step, and the default (chosen
    per step from the measured reduction), all reach the tolerance and the
    FP64 oracle's solution."""
    a, b, rho, bv = pair_from_problem(W.twosrc3d(uniform_level=4, extra_levels=2, s=0.04))
    load(a, b, rho, bv)
    a.solve(1e-12, 60)
    opts = afgpu.default_opts(rel_tol=1e-10, precision=afgpu.AFG_MIXED)
    assert opts.inner_vcycles == 0
    opts.inner_vcycles = inner
    sb = b.solve(opts)
    assert sb["rel_residual"] <= 1e-10
    assert rel_diff(b.get_solution(), a.get_solution()) <= 1e-8
    opts.inner_vcycles = 17
    with pytest.raises(afgpu.AfgError):
        b.solve(opts)


def test_empty_rhs_and_errors():
    t = afgpu.Tree(2, 8, 3)
    t.refine_uniform(2)
    with pytest.raises(afgpu.AfgError) as e:
        t.solve()
    assert e.value.code == afgpu.AFG_ERR_STATE
    z = torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda")
    t.set_rhs(z)
    st = t.solve()
    assert st["cycles"] == 1 and float(t.get_solution().abs().max()) == 0.0
    with pytest.raises(TypeError):
        t.set_rhs(z.float())
    with pytest.raises(ValueError):
        t.set_rhs(z[:-1])


@pytest.mark.parametrize("precision", [afgpu.AFG_FP64, afgpu.AFG_MIXED])
def test_graph_replay_honours_a_new_tolerance(precision):
    """Cycles replay as CUDA graphs; a later solve with a tighter tolerance must
    not reuse the earlier one (the tolerance lives in device memory)."""
    a, b, rho, bv = pair_from_problem(W.gauss2d())
    load(a, b, rho, bv)
    b.solve(afgpu.default_opts(rel_tol=1e-6, precision=precision))
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    st = b.solve(afgpu.default_opts(rel_tol=1e-11, precision=precision))
    assert st["rel_residual"] <= 1e-11
