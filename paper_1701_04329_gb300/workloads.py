"""Seeded synthetic problem set-ups shaped like the paper's workloads.

Problem definition only (sources, boundary values, refinement criteria and
the adapt-until-stable loop a user writes); none of the solver's arithmetic
lives here.  Every function works on any tree object that offers
``refine_uniform(level)``, ``cell_centers()``, ``leaf_levels()`` and
``adapt(flags, n_buf)``, so the CUDA library's tree and the test oracle are
built by the same user-side loop.

Workloads (all synthetic, the paper uses no dataset):

* ``gauss2d``  -- 2D manufactured solution u = exp(-|x-x0|^2/s^2), x0=(.5,.5),
  s=0.04, rho = Laplacian(u), Dirichlet b = u, boxes 8^2, uniform to level 4,
  refined to level 7 where |rho| h^2 > 1e-4 (the paper's Sec. 4.1 test with a
  single Gaussian).
* ``twosrc3d`` -- 3D octree, boxes 8^3, uniform 256^3 (level 6) plus two levels
  around two Gaussian sources (s=0.01, +1 at (.3,.5,.5), -1 at (.7,.5,.5)),
  u = 0 on the boundary; cells refined where |rho| > 1e-3 max|rho|.
* ``twin3d``   -- the manufactured twin of ``twosrc3d``: the same two Gaussians
  as the solution u, rho = Laplacian(u), b = u.
* ``forest2d`` -- batched: independent quadtrees with 1-4 Gaussian sources
  (s ~ U[0.01,0.08], A ~ N(0,1), centres U[0.1,0.9]^2), max level ~ U{4..9}.
* ``blobs3d``  -- 3D, uniform 128^3 plus one level where |rho| > 0.1 max|rho|,
  rho = 8 Gaussian blobs (s=0.03, A ~ N(0,1), centres U[0.15,0.85]^3).
* ``uniform3d`` -- the paper's Sec. 4.2 scaling problem: Laplacian(phi) = 1,
  phi = 0, uniform grid (512^3 in the paper).
"""
import numpy as np


def gaussian(x, c, s):
    return np.exp(-((x - np.asarray(c)) ** 2).sum(-1) / s ** 2)


def gaussian_laplacian(x, c, s):
    """Laplacian of exp(-|x-c|^2/s^2) in D = x.shape[-1] dimensions."""
    r2 = ((x - np.asarray(c)) ** 2).sum(-1)
    D = x.shape[-1]
    return (4.0 * r2 / s ** 4 - 2.0 * D / s ** 2) * np.exp(-r2 / s ** 2)


def leaf_cell_h(tree):
    lv = np.repeat(np.asarray(tree.leaf_levels()), tree.N ** tree.D)
    return 1.0 / (tree.N * 2.0 ** (lv - 1)), lv


def adapt_until_stable(tree, flag_fn, n_buf=2, max_iter=64):
    """The user's refinement loop (Sec. 2.3): evaluate the criterion on leaf
    cells, adapt, repeat until the mesh no longer changes."""
    for _ in range(max_iter):
        x = tree.cell_centers()
        h, lv = leaf_cell_h(tree)
        flags = np.asarray(flag_fn(x, h, lv), dtype=np.int8)
        flags[lv >= tree.max_level] = np.minimum(flags[lv >= tree.max_level], 0)
        if not (flags > 0).any():
            return
        added, removed = tree.adapt(flags, n_buf)
        if added == 0 and removed == 0:
            return
    raise RuntimeError("refinement did not settle")


class Problem:
    """A Poisson problem Laplacian(u) = rho on [0,1]^D with Dirichlet data."""

    def __init__(self, name, dim, box_n, uniform_level, max_level, rho, bval, flag_fn=None, u_exact=None):
        self.name, self.dim, self.box_n = name, dim, box_n
        self.uniform_level, self.max_level = uniform_level, max_level
        self.rho, self.bval, self.flag_fn, self.u_exact = rho, bval, flag_fn, u_exact

    def build(self, tree):
        tree.refine_uniform(self.uniform_level)
        if self.flag_fn is not None and self.max_level > self.uniform_level:
            adapt_until_stable(tree, self.flag_fn)
        return tree

    def data(self, tree):
        """(rho on leaf cells, Dirichlet values on leaf boundary faces)."""
        return self.rho(tree.cell_centers()), self.bval(tree.face_centers())


def gauss2d(box_n=8, uniform_level=4, max_level=7, tau=1e-4, s=0.04):
    x0 = (0.5, 0.5)
    u = lambda x: gaussian(x, x0, s)
    rho = lambda x: gaussian_laplacian(x, x0, s)
    flags = lambda x, h, lv: (np.abs(rho(x)) * h ** 2 > tau).astype(np.int8)
    return Problem("gauss2d", 2, box_n, uniform_level, max_level, rho, u, flags, u)


def _twosrc_rho(x, s=0.01):
    return gaussian(x, (0.3, 0.5, 0.5), s) - gaussian(x, (0.7, 0.5, 0.5), s)


def twosrc3d(box_n=8, uniform_level=6, extra_levels=2, s=0.01, frac=1e-3):
    rho = lambda x: _twosrc_rho(x, s)
    flags = lambda x, h, lv: (np.abs(rho(x)) > frac).astype(np.int8)
    return Problem("twosrc3d", 3, box_n, uniform_level, uniform_level + extra_levels, rho,
                   lambda x: np.zeros(len(x)), flags)


def twin3d(box_n=8, uniform_level=6, extra_levels=2, s=0.01, frac=1e-3):
    cs = [((0.3, 0.5, 0.5), 1.0), ((0.7, 0.5, 0.5), -1.0)]
    u = lambda x: sum(a * gaussian(x, c, s) for c, a in cs)
    rho = lambda x: sum(a * gaussian_laplacian(x, c, s) for c, a in cs)
    flags = lambda x, h, lv: (np.abs(_twosrc_rho(x, s)) > frac).astype(np.int8)
    return Problem("twin3d", 3, box_n, uniform_level, uniform_level + extra_levels, rho, u, flags, u)


def forest2d_params(n_trees, seed0=1000):
    """Per-tree source parameters of the batched workload."""
    out = []
    for t in range(n_trees):
        rng = np.random.default_rng(seed0 + t)
        k = int(rng.integers(1, 5))
        out.append(dict(
            centres=rng.uniform(0.1, 0.9, size=(k, 2)),
            widths=rng.uniform(0.01, 0.08, size=k),
            amps=rng.normal(0.0, 1.0, size=k),
            max_level=int(rng.integers(4, 10)),
        ))
    return out


def forest2d_problem(p, box_n=8):
    """Reading: uniform to 32^2 cells, refine where |rho| > 1e-2 max|A_k|;
    with 16^2 boxes one level less gives the same finest spacing."""
    rho = lambda x: sum(a * gaussian(x, c, s) for c, s, a in zip(p["centres"], p["widths"], p["amps"]))
    thr = 1e-2 * np.abs(p["amps"]).max()
    flags = lambda x, h, lv: (np.abs(rho(x)) > thr).astype(np.int8)
    shift = 0 if box_n == 8 else int(np.log2(box_n // 8))
    return Problem("forest2d", 2, box_n, 3 - shift, p["max_level"] - shift, rho,
                   lambda x: np.zeros(len(x)), flags)


def blobs3d(seed=1, box_n=8, uniform_level=5, n_blobs=8, s=0.03, frac=0.1):
    rng = np.random.default_rng(seed)
    cs = rng.uniform(0.15, 0.85, size=(n_blobs, 3))
    amps = rng.normal(0.0, 1.0, size=n_blobs)
    rho = lambda x: sum(a * gaussian(x, c, s) for c, a in zip(cs, amps))
    # max|rho| over the blob centres bounds the threshold from the source itself
    peak = np.abs(rho(cs)).max()
    flags = lambda x, h, lv: (np.abs(rho(x)) > frac * peak).astype(np.int8)
    return Problem("blobs3d", 3, box_n, uniform_level, uniform_level + 1, rho,
                   lambda x: np.zeros(len(x)), flags)


def uniform3d(box_n=8, level=7):
    return Problem("uniform3d", 3, box_n, level, level, lambda x: np.ones(len(x)),
                   lambda x: np.zeros(len(x)))
