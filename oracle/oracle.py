"""ctypes binding of the FP64 CPU oracle (``afmg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA library never imports it.

The oracle restates Afivo's method (Teunissen & Ebert, arXiv:1701.04329):
tree and refinement rules (Sec. 2.1-2.3), ghost cells (Sec. 2.4, 3.3),
prolongation/restriction (Sec. 2.5), red-black Gauss-Seidel (Sec. 3.1) and
the FAS V-cycle / FMG cycle (Sec. 3.2).  Array conventions (shared with the
library's public interface, not with its code):

* leaf cells: leaf boxes by level, Morton order within a level; cells of a
  box lexicographic with x fastest;
* boundary faces: leaf boxes in the same order, sides -x,+x,-y,+y(,-z,+z),
  face cells lexicographic over the tangential axes (lower axis fastest).
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "afmg_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

_lib = None


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "ot_create": (P, [I, I, I]), "ot_create_roots": (P, [I, I, I, P]), "ot_destroy": (None, [P]),
            "ot_refine_uniform": (I, [P, I]), "ot_nbox": (I, [P]), "ot_nleaf": (I, [P]),
            "ot_highest_level": (I, [P]), "ot_nleaf_cells": (LL, [P]),
            "ot_export": (None, [P, P, P, P, P, P]), "ot_cell_centers": (None, [P, P]),
            "ot_nbfaces": (LL, [P]), "ot_face_centers": (None, [P, P]),
            "ot_adapt": (I, [P, P, I, P, P]), "ot_mg_setup": (I, [P]),
            "ot_set_rhs": (None, [P, P]), "ot_set_solution": (None, [P, P]),
            "ot_get_solution": (None, [P, P]), "ot_zero_solution": (None, [P]),
            "ot_set_dirichlet": (None, [P, P]), "ot_vcycle": (None, [P, I, I, I]),
            "ot_fmg": (None, [P, I, I, I]), "ot_residual_norm": (None, [P, P, P]),
            "ot_apply_A": (None, [P, P, P]), "ot_set_homogeneous": (None, [P, I]),
            "ot_leaf_rows": (LL, [P, P, P, P]), "ot_mg_nbox": (I, [P]), "ot_mg_lmin": (I, [P]),
            "ot_mg_box_info": (None, [P, I, P]), "ot_mg_get": (None, [P, I, I, P]),
            "ot_mg_set": (None, [P, I, I, P]), "ot_fill_ghosts": (None, [P, I, I]),
            "ot_smooth": (None, [P, I, I]), "ot_gsrb_half": (None, [P, I, I]),
            "ot_restrict": (None, [P, I, I]), "ot_correct": (None, [P, I]),
            "ot_set_bc_types": (I, [P, P]), "ot_set_operator": (I, [P, I]), "ot_set_eps": (I, [P, P]),
            "ot_set_prolong": (I, [P, I]), "ot_fill_corner_ghosts": (None, [P, I, I]),
            "ot_adapt_transfer": (I, [P, P, I, I, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleTree:
    """One quadtree (D=2) or octree (D=3) with root boxes of N^D cells
    (Sec. 2.1-2.2), plus the FP64 multigrid data on it.  By default a single
    root box on [0,1]^D; roots=(rx, ry[, rz]) makes the domain a block of
    rx x ry (x rz) unit root boxes, [0,rx] x [0,ry] (x [0,rz])."""

    def __init__(self, dim, box_n, max_level, roots=None):
        self.D, self.N, self.max_level = dim, box_n, max_level
        self.roots = tuple(int(r) for r in roots) if roots is not None else (1,) * dim
        if len(self.roots) != dim:
            raise ValueError("roots needs one count per axis")
        nr = np.array(list(self.roots) + [1] * (3 - dim), np.int32)
        self._h = lib().ot_create_roots(dim, box_n, max_level, _p(nr))
        if not self._h:
            raise ValueError("bad tree parameters")
        self._mg = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ot_destroy(h)
            self._h = None

    # ---- tree --------------------------------------------------------------
    def refine_uniform(self, level):
        if lib().ot_refine_uniform(self._h, level) != 0:
            raise ValueError("refine_uniform failed")
        self._mg = False

    @property
    def nbox(self):
        return lib().ot_nbox(self._h)

    @property
    def nleaf(self):
        return lib().ot_nleaf(self._h)

    @property
    def highest_level(self):
        return lib().ot_highest_level(self._h)

    @property
    def n_leaf_cells(self):
        return lib().ot_nleaf_cells(self._h)

    @property
    def n_bfaces(self):
        return lib().ot_nbfaces(self._h)

    def export(self):
        n, D = self.nbox, self.D
        level = np.zeros(n, np.int32)
        idx = np.zeros((n, D), np.int32)
        parent = np.zeros(n, np.int32)
        children = np.zeros((n, 2 ** D), np.int32)
        nbs = np.zeros((n, 3 ** D - 1), np.int32)
        lib().ot_export(self._h, _p(level), _p(idx), _p(parent), _p(children), _p(nbs))
        return dict(level=level, idx=idx, parent=parent, children=children, neighbours=nbs)

    def leaf_levels(self):
        e = self.export()
        return e["level"][e["children"][:, 0] < 0]

    def cell_centers(self):
        x = np.zeros((self.n_leaf_cells, self.D))
        lib().ot_cell_centers(self._h, _p(x))
        return x

    def face_centers(self):
        x = np.zeros((self.n_bfaces, self.D))
        lib().ot_face_centers(self._h, _p(x))
        return x

    def adapt(self, flags, n_buf=2):
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.size == self.n_leaf_cells
        a, r = ctypes.c_int(0), ctypes.c_int(0)
        rc = lib().ot_adapt(self._h, _p(flags), n_buf, ctypes.byref(a), ctypes.byref(r))
        if rc != 0:
            raise RuntimeError("adapt failed (%d)" % rc)
        self._mg = False
        return a.value, r.value

    def adapt_transfer(self, flags, u, n_buf=2, scheme=0):
        """adapt() that carries the leaf field u along: kept leaves copy,
        derefined parents average their children, new children are prolonged
        (scheme 0 linear, 1 bi/trilinear, 2 copy).  Returns (u_new, added,
        removed); the stored solution is overwritten."""
        self._need_mg()
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert flags.size == self.n_leaf_cells and u.size == self.n_leaf_cells
        # the adapted tree has at most 2^D times the leaves
        out = np.zeros(self.n_leaf_cells * 2 ** self.D)
        a, r = ctypes.c_int(0), ctypes.c_int(0)
        rc = lib().ot_adapt_transfer(self._h, _p(flags), n_buf, scheme, _p(u), _p(out), ctypes.byref(a),
                                     ctypes.byref(r))
        if rc != 0:
            raise RuntimeError("adapt_transfer failed (%d)" % rc)
        self._mg = False
        return out[:self.n_leaf_cells].copy(), a.value, r.value

    # ---- multigrid data ----------------------------------------------------
    def _need_mg(self):
        if not self._mg:
            if lib().ot_mg_setup(self._h) != 0:
                raise RuntimeError("mg setup failed")
            self._mg = True

    def set_rhs(self, rho):
        self._need_mg()
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.size == self.n_leaf_cells
        lib().ot_set_rhs(self._h, _p(rho))

    def set_dirichlet(self, b):
        self._need_mg()
        b = np.ascontiguousarray(b, dtype=np.float64)
        assert b.size == self.n_bfaces
        lib().ot_set_dirichlet(self._h, _p(b))

    def set_solution(self, u):
        self._need_mg()
        u = np.ascontiguousarray(u, dtype=np.float64)
        lib().ot_set_solution(self._h, _p(u))

    def zero_solution(self):
        self._need_mg()
        lib().ot_zero_solution(self._h)

    def get_solution(self):
        u = np.zeros(self.n_leaf_cells)
        lib().ot_get_solution(self._h, _p(u))
        return u

    def set_boundary_types(self, types):
        """Per domain side (-x,+x,-y,+y[,-z,+z]): 0 Dirichlet, 1 Neumann, 2 periodic
        (both sides of an axis; switched only while the tree is its root boxes alone)."""
        t = np.ascontiguousarray(types, dtype=np.int32)
        assert t.size == 2 * self.D
        if lib().ot_set_bc_types(self._h, _p(t)) != 0:
            raise ValueError("boundary types: 0/1/2, periodic in pairs and set on the root boxes alone, "
                             "at least one Dirichlet side")
        self.bc_types = [int(v) for v in t]

    def set_operator(self, op):
        """0: Laplacian; 1: div(eps grad u) with harmonic-mean face
        coefficients (Sec. 3.4); 2: the same in (r,z) coordinates, r = x (2D)."""
        if lib().ot_set_operator(self._h, int(op)) != 0:
            raise ValueError("operator: 0, 1, or 2 (2D only)")
        self.op = int(op)

    def set_eps(self, eps):
        """Coefficient per leaf cell (> 0), canonical order; coarse levels take
        the mean of their children.  Set again after every change of the tree."""
        self._need_mg()
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        assert eps.size == self.n_leaf_cells
        if lib().ot_set_eps(self._h, _p(eps)) != 0:
            raise ValueError("eps must be positive")
        self.eps = eps.copy()

    def set_prolong(self, scheme):
        """Prolongation of the coarse-grid correction: 0 linear (1/2,1/4,1/4)
        / (1/4,...) (default), 1 bilinear / trilinear, 2 zeroth order."""
        if lib().ot_set_prolong(self._h, int(scheme)) != 0:
            raise ValueError("prolongation: 0, 1 or 2")

    def fill_corner_ghosts(self, level, which=0):
        lib().ot_fill_corner_ghosts(self._h, level, which)

    def set_homogeneous(self, hom):
        self._need_mg()
        lib().ot_set_homogeneous(self._h, int(hom))

    def vcycle(self, n_down=2, n_up=2, n_base=4):
        self._need_mg()
        lib().ot_vcycle(self._h, n_down, n_up, n_base)

    def fmg(self, n_down=2, n_up=2, n_base=4):
        self._need_mg()
        lib().ot_fmg(self._h, n_down, n_up, n_base)

    def residual_norm(self):
        """(max_leaf |rho - A u|, max_leaf |rho|), composite operator."""
        self._need_mg()
        r, p = ctypes.c_double(0), ctypes.c_double(0)
        lib().ot_residual_norm(self._h, ctypes.byref(r), ctypes.byref(p))
        return r.value, p.value

    def solve(self, rel_tol=1e-10, max_cycles=50, n_down=2, n_up=2, n_base=4, history=None):
        """FMG (cycle 1) then V-cycles until max|r|/max|rho| <= rel_tol.
        Returns the number of cycles."""
        self.fmg(n_down, n_up, n_base)
        cycles = 1
        while True:
            r, p = self.residual_norm()
            rel = r / p if p > 0 else r
            if history is not None:
                history.append(rel)
            if rel <= rel_tol or cycles >= max_cycles:
                return cycles
            self.vcycle(n_down, n_up, n_base)
            cycles += 1

    def apply_A(self, u):
        """Composite operator A(u) on leaf data, boundary data included.
        Overwrites the stored solution."""
        self._need_mg()
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(self.n_leaf_cells)
        lib().ot_apply_A(self._h, _p(u), _p(out))
        return out

    def leaf_rows(self):
        """Sparse matrix K of the composite operator on leaf cells (boundary
        data excluded), assembled from the oracle's ghost rules."""
        import scipy.sparse as sp
        self._need_mg()
        n = lib().ot_leaf_rows(self._h, None, None, None)
        row = np.zeros(n, np.int32)
        col = np.zeros(n, np.int32)
        val = np.zeros(n)
        lib().ot_leaf_rows(self._h, _p(row), _p(col), _p(val))
        m = self.n_leaf_cells
        return sp.csr_matrix((val, (row, col)), shape=(m, m))

    # ---- low-level access for unit tests ------------------------------------
    def mg_boxes(self):
        self._need_mg()
        n = lib().ot_mg_nbox(self._h)
        out = []
        for b in range(n):
            info = np.zeros(20, np.int32)
            lib().ot_mg_box_info(self._h, b, _p(info))
            out.append(dict(level=int(info[0]), M=int(info[1]), tbox=int(info[2]), parent=int(info[3]),
                            refined=bool(info[4]), kind=info[5:11].copy(), nbid=info[11:17].copy(),
                            poff=info[17:20].copy()))
        return out

    @property
    def lmin(self):
        self._need_mg()
        return lib().ot_mg_lmin(self._h)

    def mg_get(self, b, var, M):
        a = np.zeros((M + 2) ** self.D)
        lib().ot_mg_get(self._h, b, var, _p(a))
        return a.reshape((M + 2,) * self.D)  # index [k][j][i] (3D) or [j][i]

    def mg_set(self, b, var, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        lib().ot_mg_set(self._h, b, var, _p(a))

    def fill_ghosts(self, level, which=0):
        lib().ot_fill_ghosts(self._h, level, which)

    def smooth(self, level, n):
        lib().ot_smooth(self._h, level, n)

    def gsrb_half(self, level, colour):
        lib().ot_gsrb_half(self._h, level, colour)

    def restrict(self, level, which=0):
        lib().ot_restrict(self._h, level, which)

    def correct(self, level):
        lib().ot_correct(self._h, level)
