"""Boundary calls beyond the solve, on the GPU: device memory from a caller's
allocator (PyTorch's caching allocator through afg_set_allocator) gives the
same solution bit for bit, and the device form of the cell centres equals
the host form."""
import numpy as np
import pytest

from paper_1701_04329_gb300 import afgpu
from paper_1701_04329_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(p, prec):
    t = afgpu.Tree(p.dim, p.box_n, p.max_level)
    p.build(t)
    rho, b = p.data(t)
    t.set_rhs(torch.tensor(rho, device="cuda"))
    t.set_dirichlet(torch.tensor(b, device="cuda"))
    t.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
    st = t.solve(afgpu.default_opts(rel_tol=1e-10, precision=prec))
    return t, t.get_solution().clone(), st


@pytest.mark.parametrize("prec", [afgpu.AFG_FP64, afgpu.AFG_MIXED])
def test_torch_caching_allocator_gives_the_same_solve(prec):
    p = W.gauss2d(max_level=6)
    t0, u0, st0 = _solve(p, prec)
    t0.close()
    seen = []

    def alloc(n):
        ptr = torch.cuda.caching_allocator_alloc(n)
        seen.append(n)
        return ptr

    afgpu.set_allocator(alloc, torch.cuda.caching_allocator_delete)
    try:
        t1, u1, st1 = _solve(p, prec)
        assert len(seen) > 0
        assert st1["cycles"] == st0["cycles"]
        assert torch.equal(u0, u1)
        t1.close()
    finally:
        afgpu.set_allocator(None, None)
    torch.cuda.synchronize()


def test_allocator_returning_null_is_reported_as_out_of_memory():
    p = W.gauss2d(max_level=5)
    afgpu.set_allocator(lambda n: 0, lambda ptr: None)
    try:
        t = afgpu.Tree(p.dim, p.box_n, p.max_level)
        p.build(t)
        with pytest.raises(afgpu.AfgError) as e:
            t.set_rhs(torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda"))
        assert e.value.code == afgpu.AFG_ERR_NOMEM
    finally:
        afgpu.set_allocator(None, None)


@pytest.mark.parametrize("D,roots", [(2, None), (3, None), (2, (3, 2))])
def test_cell_centres_on_the_device_equal_the_host_ones(D, roots):
    t = afgpu.Tree(D, 8, 4, roots=roots)
    t.refine_uniform(2)
    rng = np.random.default_rng(5)
    t.adapt(np.repeat((rng.random(t.info().n_leaves) < 0.4).astype(np.int8), 8 ** D), 1)
    host = t.cell_centers()
    dev = t.cell_centers_device().cpu().numpy()
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("D,N", [(2, 8), (2, 16), (3, 8)])
def test_threads_per_box_choices_give_the_same_mixed_solve(D, N):
    """The FP32 half-sweep with half the threads per box (two vectors per
    thread) computes the same cells from the same staged data: the mixed
    solve is bit for bit the same; other values are refused."""
    from tests.gpu_helpers import pair_random
    _, b, rho, bv = pair_random(D, N, 2, 1, 40 + N)
    b.set_rhs(torch.tensor(rho, device="cuda"))
    b.set_dirichlet(torch.tensor(bv, device="cuda"))
    nv = min((N ** D // 2) // 4, 256)
    sols = []
    for tpb in (0, nv, nv // 2):
        b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))
        st = b.solve(afgpu.default_opts(rel_tol=1e-10, precision=afgpu.AFG_MIXED, threads_per_box=tpb))
        sols.append((st["cycles"], b.get_solution().clone()))
    assert sols[0][0] == sols[1][0] == sols[2][0]
    assert torch.equal(sols[0][1], sols[1][1]) and torch.equal(sols[0][1], sols[2][1])
    with pytest.raises(afgpu.AfgError) as e:
        b.solve(afgpu.default_opts(rel_tol=1e-10, precision=afgpu.AFG_MIXED, threads_per_box=nv + 1))
    assert e.value.code == afgpu.AFG_ERR_ARG
