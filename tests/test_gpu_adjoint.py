"""GPU adjoint (transposed-operator kernel + preconditioned BiCGStab through
the C ABI) against the oracle: direct sparse solve of K^T on small trees,
the oracle's own BiCGStab, the uniform-grid symmetric case, and central
finite differences of a quadratic loss through torch.autograd."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import composite
from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W
from tests.gpu_helpers import pair_random, pair_from_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 4, 2, 2, 51), (2, 8, 1, 3, 52), (3, 4, 1, 2, 53),
                                               (3, 8, 1, 2, 54)])
def test_adjoint_matches_transpose_solve(D, N, uni, extra, seed):
    a, b, rho, bv = pair_random(D, N, uni, extra, seed)
    g = np.random.default_rng(seed).normal(size=a.n_leaf_cells)
    ref = oadj.direct(a, g)
    lam, db, st = b.adjoint(torch.tensor(g, device="cuda"), afgpu.default_opts(rel_tol=1e-12, max_cycles=100))
    assert st["rel_residual"] <= 1e-12
    lam = lam.cpu().numpy()
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()
    dref = oadj.dl_db(a, ref)
    assert np.abs(db.cpu().numpy() - dref).max() <= 1e-9 * np.abs(dref).max()
    # the oracle's own BiCGStab lands on the same vector
    lo, _ = oadj.bicgstab(a, g, tol=1e-12)
    assert np.abs(lam - lo).max() <= 1e-9 * np.abs(lo).max()


@pytest.mark.parametrize("D,N,uni,extra,seed", [(2, 8, 1, 3, 55), (3, 8, 1, 2, 56)])
def test_adjoint_with_fp32_preconditioner(D, N, uni, extra, seed):
    """AFG_MIXED: the preconditioner's V-cycle in FP32, K^T and the
    BiCGStab recurrences in FP64 -- the same lambda at the same FP64
    tolerance."""
    a, b, rho, bv = pair_random(D, N, uni, extra, seed)
    g = np.random.default_rng(seed).normal(size=a.n_leaf_cells)
    ref = oadj.direct(a, g)
    lam, db, st = b.adjoint(torch.tensor(g, device="cuda"),
                            afgpu.default_opts(rel_tol=1e-12, max_cycles=100, precision=afgpu.AFG_MIXED))
    assert st["rel_residual"] <= 1e-12
    assert np.abs(lam.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
    dref = oadj.dl_db(a, ref)
    assert np.abs(db.cpu().numpy() - dref).max() <= 1e-9 * np.abs(dref).max()


def test_uniform_adjoint_equals_forward_solve():
    """On a uniform tree K is symmetric: K^T lam = g is the forward problem
    with rho = g and b = 0."""
    t = afgpu.Tree(3, 8, 3)
    t.refine_uniform(3)
    g = torch.tensor(np.random.default_rng(55).normal(size=t.n_leaf_cells), device="cuda")
    lam, _, _ = t.adjoint(g, afgpu.default_opts(rel_tol=1e-13, max_cycles=100))
    t.set_rhs(g)
    t.set_dirichlet(torch.zeros(t.n_bfaces, dtype=torch.float64, device="cuda"))
    t.set_solution(torch.zeros_like(g))
    t.solve(afgpu.default_opts(rel_tol=1e-13, max_cycles=60))
    u = t.get_solution()
    assert float((lam - u).abs().max()) <= 1e-9 * float(u.abs().max())


def test_autograd_gradient_vs_central_differences():
    """L = 1/2 sum_leaves vol (u - u*)^2 is quadratic in (rho, b): central
    differences are exact up to round-off and the solve tolerance."""
    from paper_1701_04329_gb300.autograd import PoissonSolve
    p = W.blobs3d(uniform_level=3)
    t = afgpu.Tree(3, 8, p.max_level)
    p.build(t)
    rho_h, b_h = p.data(t)
    rng = np.random.default_rng(3)
    e = t.export()
    vol = torch.tensor(composite.cell_volumes(3, 8, e["level"], e["children"]), device="cuda")
    ustar = torch.tensor(W.blobs3d(seed=2, uniform_level=3).rho(t.cell_centers()) * 1e-4, device="cuda")
    opts = afgpu.default_opts(rel_tol=1e-12, max_cycles=80)
    # the adjoint's relative residual floor depends on g's dynamic range; 1e-11
    # keeps the gradient error far below the 1e-6 of the comparison
    adj = afgpu.default_opts(rel_tol=1e-11, max_cycles=200)
    rho = torch.tensor(rho_h, device="cuda", requires_grad=True)
    b = torch.tensor(rng.normal(scale=1e-3, size=t.n_bfaces), device="cuda", requires_grad=True)

    def loss(r, bb):
        u = PoissonSolve.apply(r, bb, t, opts, adj)
        return 0.5 * (vol * (u - ustar) ** 2).sum()

    L = loss(rho, b)
    L.backward()
    gr, gb = rho.grad.clone(), b.grad.clone()
    for i in rng.choice(t.n_leaf_cells, 20, replace=False):
        h = 1e-6 * max(1.0, abs(float(rho.detach()[i])))
        with torch.no_grad():
            rp = rho.detach().clone(); rp[i] += h
            rm = rho.detach().clone(); rm[i] -= h
            fd = (float(loss(rp, b.detach())) - float(loss(rm, b.detach()))) / (2 * h)
        assert abs(fd - float(gr[i])) <= 1e-6 * float(gr.abs().max()) + 1e-6 * abs(fd)
    for f in rng.choice(t.n_bfaces, 20, replace=False):
        h = 1e-6
        with torch.no_grad():
            bp = b.detach().clone(); bp[f] += h
            bm = b.detach().clone(); bm[f] -= h
            fd = (float(loss(rho.detach(), bp)) - float(loss(rho.detach(), bm))) / (2 * h)
        assert abs(fd - float(gb[f])) <= 1e-6 * float(gb.abs().max()) + 1e-6 * abs(fd)
