"""The allocation-free residual-norm entry point, through the C ABI.

afg_forest_residual_norms_noalloc serves callers that cannot allocate device
memory where they check convergence (a framework that owns the whole device
pool, or a loop that cannot afford cudaMalloc's implicit synchronisation).
It must return the same per-tree norms as the allocating path --
afg_forest_solve's reported norms, and afg_residual_norm on each tree holding
the forest's solution -- on two calls in a row (its scratch array keeps the previous
call's contents), and reject forests larger than its fixed scratch."""
import numpy as np
import pytest

from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _trees(n):
    out = []
    for prm in W.forest2d_params(n, seed0=2000):
        p = W.forest2d_problem(dict(prm, max_level=min(prm["max_level"], 6)))
        t = afgpu.Tree(2, 8, p.max_level)
        p.build(t)
        rho, b = p.data(t)
        out.append((t, rho, b))
    return out


def test_noalloc_norms_equal_the_allocating_path_on_two_calls():
    items = _trees(6)
    f = afgpu.Forest([t for t, _, _ in items])
    f.set_rhs(torch.tensor(np.concatenate([r for _, r, _ in items]), device="cuda"))
    f.set_dirichlet(torch.tensor(np.concatenate([b for _, _, b in items]), device="cuda"))
    opts = afgpu.default_opts(rel_tol=1e-10)
    stats = f.solve(opts)
    solver_r = np.array([s["max_residual"] for s in stats])
    solver_p = np.array([s["max_rho"] for s in stats])
    tol = 1e-12
    for _ in range(2):
        r, p = f.residual_norms_noalloc()
        assert np.all(np.abs(r - solver_r) <= tol * np.abs(solver_r) + 1e-300)
        assert np.all(np.abs(p - solver_p) <= tol * np.abs(solver_p))
    # each tree given the forest's solution and measured with afg_residual_norm
    # (a tree of one root box solves its level 2 in the bottom launch, so a
    # solve of its own rounds differently from the forest's; the same u must
    # give the same norms)
    u = f.get_solution()
    off = 0
    for k, (t, rho, b) in enumerate(items):
        n = len(rho)
        t.set_rhs(torch.tensor(rho, device="cuda"))
        t.set_dirichlet(torch.tensor(b, device="cuda"))
        t.set_solution(u[off:off + n].clone())
        off += n
        tr, tp = t.residual_norm()
        assert abs(r[k] - tr) <= tol * abs(tr) and abs(p[k] - tp) <= tol * abs(tp)


def test_noalloc_rejects_forests_beyond_its_scratch():
    trees = []
    for _ in range(1025):
        t = afgpu.Tree(2, 4, 1)
        trees.append(t)
    f = afgpu.Forest(trees)
    with pytest.raises(afgpu.AfgError) as e:
        f.residual_norms_noalloc()
    assert e.value.code == afgpu.AFG_ERR_ARG
    assert "1024" in str(e.value)
