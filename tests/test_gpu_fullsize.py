"""Parity at the benchmark sizes, in the launch configuration bench.py times.

* 3D two-source workload (17.6 M unknowns): FP64 GPU solve vs the oracle
  after the same cycle count (element by element, 1e-12 relative), and the
  mixed-precision solve at 1e-8 against it.
* Differentiable 3D workload (128^3 + 1 level): gradients of a quadratic loss
  through torch.autograd against central finite differences (step 1e-6) on
  20 random cells and 20 boundary faces (seed 3).  The loss is quadratic, so
  the differences are exact up to the forward solves' tolerance (1e-12
  relative residual): the bound is 1e-5 of the largest gradient entry."""
import numpy as np
import pytest

from oracle.oracle import OracleTree
from oracle import composite
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import rel_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_twosrc3d_full_size_fp64_and_mixed():
    p = W.twosrc3d()
    a = OracleTree(3, 8, p.max_level)
    b = afgpu.Tree(3, 8, p.max_level)
    p.build(a)
    p.build(b)
    assert a.n_leaf_cells == b.n_leaf_cells == 17637376
    rho, bv = p.data(a)
    a.set_rhs(rho); a.set_dirichlet(bv); a.zero_solution()
    hist = []
    ca = a.solve(1e-8, 40, history=hist)
    uref = a.get_solution()
    rho_d, b_d = torch.tensor(rho, device="cuda"), torch.tensor(bv, device="cuda")
    b.set_rhs(rho_d); b.set_dirichlet(b_d); b.set_solution(torch.zeros_like(rho_d))
    st = b.solve(afgpu.default_opts(rel_tol=1e-8))
    assert st["cycles"] == ca
    assert rel_diff(b.get_solution(), uref) <= 1e-12
    assert np.allclose(st["history"][:len(hist)], hist, rtol=1e-6, atol=1e-12)
    # mixed precision: same tolerance, solution within the FP64 one's accuracy
    b.set_solution(torch.zeros_like(rho_d))
    sm = b.solve(afgpu.default_opts(rel_tol=1e-8, precision=afgpu.AFG_MIXED))
    assert sm["rel_residual"] <= 1e-8
    # both solutions carry an error of order tol * cond from the exact composite
    # solution; tighten both and compare at 1e-8
    b.set_solution(torch.zeros_like(rho_d))
    b.solve(afgpu.default_opts(rel_tol=1e-12, precision=afgpu.AFG_MIXED, max_cycles=60))
    um = b.get_solution()
    a.zero_solution()
    a.solve(1e-12, 60)
    assert rel_diff(um, a.get_solution()) <= 1e-8


def test_blobs3d_full_size_gradient_vs_finite_differences():
    from paper_1701_04329_gb300.autograd import PoissonSolve
    p = W.blobs3d()
    t = afgpu.Tree(3, 8, p.max_level)
    p.build(t)
    e = t.export()
    vol = torch.tensor(composite.cell_volumes(3, 8, e["level"], e["children"]), device="cuda")
    rho_h, b_h = p.data(t)
    x = t.cell_centers()
    ustar = torch.tensor(1e-4 * W.blobs3d(seed=2).rho(x), device="cuda")
    rng = np.random.default_rng(3)
    opts = afgpu.default_opts(rel_tol=1e-12, max_cycles=80)
    # the adjoint's relative residual floor depends on g's dynamic range; 1e-11
    # keeps the gradient error far below the 1e-6 of the comparison
    adj = afgpu.default_opts(rel_tol=1e-11, max_cycles=200)
    rho = torch.tensor(rho_h, device="cuda", requires_grad=True)
    b = torch.tensor(rng.normal(scale=1e-3, size=t.n_bfaces), device="cuda", requires_grad=True)

    def loss(r, bb):
        u = PoissonSolve.apply(r, bb, t, opts, adj)
        return 0.5 * (vol * (u - ustar) ** 2).sum()

    loss(rho, b).backward()
    gr, gb = rho.grad.clone(), b.grad.clone()
    r0, b0 = rho.detach().clone(), b.detach().clone()
    for i in rng.choice(t.n_leaf_cells, 20, replace=False):
        h = 1e-6 * max(1.0, abs(float(r0[i])))
        rp, rm = r0.clone(), r0.clone()
        rp[i] += h
        rm[i] -= h
        with torch.no_grad():
            fd = (float(loss(rp, b0)) - float(loss(rm, b0))) / (2 * h)
        assert abs(fd - float(gr[i])) <= 1e-5 * float(gr.abs().max())
    for f in rng.choice(t.n_bfaces, 20, replace=False):
        h = 1e-6
        bp, bm = b0.clone(), b0.clone()
        bp[f] += h
        bm[f] -= h
        with torch.no_grad():
            fd = (float(loss(r0, bp)) - float(loss(r0, bm))) / (2 * h)
        assert abs(fd - float(gb[f])) <= 1e-5 * float(gb.abs().max())
