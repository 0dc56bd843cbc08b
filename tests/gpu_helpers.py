"""Shared set-up for the GPU parity tests: the same problem on the oracle and
on the library, from the same seeded inputs."""
import numpy as np

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import afgpu


def pair_from_problem(p):
    a = OracleTree(p.dim, p.box_n, p.max_level)
    b = afgpu.Tree(p.dim, p.box_n, p.max_level)
    p.build(a)
    p.build(b)
    rho, bv = p.data(a)
    return a, b, rho, bv


def pair_random(D, N, uniform, extra, seed, frac=0.35, n_buf=1):
    rng = np.random.default_rng(seed)
    a = OracleTree(D, N, uniform + extra)
    b = afgpu.Tree(D, N, uniform + extra)
    for t in (a, b):
        t.refine_uniform(uniform)
    for _ in range(extra):
        flags = np.repeat((rng.random(a.nleaf) < frac).astype(np.int8), N ** D)
        a.adapt(flags, n_buf)
        b.adapt(flags, n_buf)
    x = a.cell_centers()
    rho = np.sin(5 * x[:, 0] + 1) * np.cos(3 * x[:, 1]) + rng.normal(scale=0.1, size=len(x))
    bv = rng.normal(size=a.n_bfaces)
    return a, b, rho, bv


def load(a, b, rho, bv):
    import torch
    a.set_rhs(rho)
    a.set_dirichlet(bv)
    a.zero_solution()
    b.set_rhs(torch.tensor(rho, device="cuda"))
    if len(bv):
        b.set_dirichlet(torch.tensor(bv, device="cuda"))
    b.set_solution(torch.zeros(len(rho), dtype=torch.float64, device="cuda"))


def rel_diff(u_gpu, u_ref):
    u = u_gpu.cpu().numpy() if hasattr(u_gpu, "cpu") else u_gpu
    return np.abs(u - u_ref).max() / max(np.abs(u_ref).max(), 1e-300)
