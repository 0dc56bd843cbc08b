"""FP64 adjoint of the composite solve -- TEST INFRASTRUCTURE ONLY.

Not in the paper (an addition): for a loss L(u) with u = A^-1(rho, b), the
gradient is lam = K^-T dL/du (K = the composite leaf operator, Sec. 3.2-3.3)
and dL/db_f = -(2/h^2) lam_i(f) on Dirichlet sides (ghost 2b - u), -(1/h) lam_i(f)
on Neumann sides (ghost u + h b).  K is not symmetric
on refined trees (the conservative refinement-boundary ghosts couple fine to
coarse with 1/2 but coarse to fine through the mean of the children), so the
true transpose is needed.  Two solvers:

* direct(): scipy sparse LU of K^T (the definition, for small trees);
* bicgstab(): BiCGStab (van der Vorst 1992) with right preconditioner
  W M W^-1, M = one oracle V-cycle from zero with homogeneous boundary data,
  W = diag(cell volumes, times r in (r,z)) -- W K is symmetric up to the
  refinement-boundary terms, so W M W^-1 approximates K^-T.

With a variable coefficient (Sec. 3.4-3.5) the face terms carry the face
coefficients, and dL/db_f takes them too (-B^T lam with B of that operator).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import composite


def operator(tree):
    """(K, B) of the tree's composite system: the Laplacian's rows from the
    oracle's ghost rules, or the geometric assembly of a variable-coefficient
    operator (Sec. 3.4-3.5) with the coefficient last set on the tree."""
    e = tree.export()
    bct = getattr(tree, "bc_types", None)
    roots = getattr(tree, "roots", None)
    op = getattr(tree, "op", 0)
    if op == 0:
        _, B = composite.assemble(tree.D, tree.N, e["level"], e["idx"], e["children"], bct, roots=roots)
        return tree.leaf_rows(), B
    return composite.assemble_var(tree.D, tree.N, e["level"], e["idx"], e["children"], tree.eps, op, bct,
                                  roots=roots)


def weights(tree):
    """Cell volumes; in (r,z) times r (the finite-volume weights)."""
    e = tree.export()
    w = composite.cell_volumes(tree.D, tree.N, e["level"], e["children"])
    if getattr(tree, "op", 0) == 2:
        w = w * tree.cell_centers()[:, 0]
    return w


def direct(tree, g):
    K, _ = operator(tree)
    return spla.spsolve(K.T.tocsc(), g)


def dl_db(tree, lam):
    _, B = operator(tree)
    return -(B.T @ lam)


def bicgstab(tree, g, tol=1e-12, maxit=100, n_down=2, n_up=2, n_base=4):
    """The tree's rhs/solution/boundary data are overwritten."""
    KT = operator(tree)[0].T.tocsr()
    w = weights(tree)
    tree.set_dirichlet(np.zeros(tree.n_bfaces))
    tree.set_homogeneous(1)

    def P(r):
        tree.set_rhs(r / w)
        tree.zero_solution()
        tree.vcycle(n_down, n_up, n_base)
        return w * tree.get_solution()

    b = np.asarray(g, dtype=np.float64)
    bn = np.abs(b).max()
    x = np.zeros_like(b)
    if bn == 0:
        return x, 0
    r = b.copy()
    rh = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_old = alpha = omega = 1.0
    it = 0
    for it in range(1, maxit + 1):
        rho_new = rh @ r
        beta = (rho_new / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = P(p)
        v = KT @ ph
        alpha = rho_new / (rh @ v)
        s = r - alpha * v
        if np.abs(s).max() / bn <= tol:
            x += alpha * ph
            break
        sh = P(s)
        t = KT @ sh
        omega = (t @ s) / (t @ t)
        x += alpha * ph + omega * sh
        r = s - omega * t
        if np.abs(r).max() / bn <= tol:
            break
        rho_old = rho_new
    tree.set_homogeneous(0)
    return x, it
