"""Differentiable Poisson solve on an AMR tree (torch.autograd).

Forward: the FAS multigrid solve of the library (arXiv:1701.04329 Sec. 3).
Backward (an addition to the paper): the library's adjoint solve
K^T lam = dL/du for the transposed composite operator; dL/drho = lam and
dL/db = -(2/h^2) lam (Dirichlet side) or -(1/h) lam (Neumann side) at the
cell next to each boundary face.
"""
import torch

from . import afgpu


class PoissonSolve(torch.autograd.Function):
    """u = PoissonSolve.apply(rho, b, tree, opts, adj_opts): rho on leaf cells,
    b on leaf boundary faces (canonical orders, float64 CUDA tensors); opts
    control the forward solve, adj_opts (default: opts) the adjoint solve."""

    @staticmethod
    def forward(ctx, rho, b, tree, opts=None, adj_opts=None):
        opts = opts or afgpu.default_opts()
        tree.set_rhs(rho.detach().contiguous())
        if b.numel():
            tree.set_dirichlet(b.detach().contiguous())
        tree.set_solution(torch.zeros_like(rho))
        tree.solve(opts)
        ctx.tree, ctx.opts, ctx.nb = tree, adj_opts or opts, b.numel()
        return tree.get_solution()

    @staticmethod
    def backward(ctx, gu):
        lam, db, _ = ctx.tree.adjoint(gu.detach().contiguous(), ctx.opts)
        return lam, db[: ctx.nb], None, None, None
