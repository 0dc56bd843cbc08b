"""Python binding of libafgpu (``include/afgpu.h``): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; torch supplies
device memory and the current stream.  There is no fallback: if the
compiled library is missing, importing the binding raises.

Method: Teunissen & Ebert, "Afivo" (arXiv:1701.04329): quadtree/octree AMR
(Sec. 2), FAS multigrid with red-black Gauss-Seidel (Sec. 3).
"""
import ctypes
import os

import numpy as np

from . import build as _build

AFG_OK, AFG_ERR_ARG, AFG_ERR_CUDA, AFG_ERR_NOMEM, AFG_ERR_STATE, AFG_ERR_NOT_CONVERGED, AFG_ERR_TIMEOUT = (
    0, -1, -2, -3, -4, -5, -6)
AFG_BC_DIRICHLET, AFG_BC_NEUMANN, AFG_BC_PERIODIC = 0, 1, 2
AFG_FP64, AFG_MIXED = 0, 1
AFG_OP_LAPLACE, AFG_OP_VAR, AFG_OP_VAR_RZ = 0, 1, 2
AFG_PROLONG_LINEAR, AFG_PROLONG_MULTILINEAR, AFG_PROLONG_ZEROTH = 0, 1, 2


class AfgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("afgpu error %d: %s" % (code, msg))
        self.code = code


class MgOpts(ctypes.Structure):
    _fields_ = [("n_down", ctypes.c_int), ("n_up", ctypes.c_int), ("n_base", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("rel_tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("inner_vcycles", ctypes.c_int), ("use_graph", ctypes.c_int), ("threads_per_box", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("rel_residual", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("max_rho", ctypes.c_double), ("seconds", ctypes.c_double), ("history", ctypes.c_double * 64)]

    def as_dict(self):
        n = min(self.cycles, 64)
        return dict(cycles=self.cycles, rel_residual=self.rel_residual, max_residual=self.max_residual,
                    max_rho=self.max_rho, seconds=self.seconds, history=list(self.history[:max(n, 1)]))


class TreeInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("box_n", ctypes.c_int), ("max_level", ctypes.c_int),
                ("highest_level", ctypes.c_int), ("n_boxes", ctypes.c_int), ("n_leaves", ctypes.c_int),
                ("n_leaf_cells", ctypes.c_longlong), ("n_bfaces", ctypes.c_longlong),
                ("boxes_per_level", ctypes.c_int * 32), ("leaves_per_level", ctypes.c_int * 32)]


_LIB = None
P, I, LL, DBL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
_SIGS = {
    "afg_default_opts": (None, [P]), "afg_last_error": (ctypes.c_char_p, []),
    "afg_tree_create": (I, [I, I, I, P]), "afg_tree_create_roots": (I, [I, I, I, P, P]),
    "afg_tree_destroy": (I, [P]), "afg_set_stream": (I, [P, P]),
    "afg_refine_uniform": (I, [P, I]), "afg_cell_centers": (I, [P, P]), "afg_face_centers": (I, [P, P]),
    "afg_leaf_levels": (I, [P, P]), "afg_adapt": (I, [P, P, I, P, P]), "afg_info": (I, [P, P]),
    "afg_export_tree": (I, [P, P, P, P, P, P]), "afg_set_rhs": (I, [P, P]), "afg_set_dirichlet": (I, [P, P]),
    "afg_set_boundary_types": (I, [P, P]),
    "afg_set_solution": (I, [P, P]), "afg_get_solution": (I, [P, P]), "afg_fmg": (I, [P, P, P]),
    "afg_vcycle": (I, [P, P, P]), "afg_solve": (I, [P, P, P]), "afg_residual_norm": (I, [P, P, P]),
    "afg_adjoint": (I, [P, P, P, P, P, P]), "afg_forest_create": (I, [I, P, P]), "afg_forest_destroy": (I, [P]),
    "afg_forest_set_stream": (I, [P, P]), "afg_forest_counts": (I, [P, P, P]), "afg_forest_set_rhs": (I, [P, P]),
    "afg_forest_set_dirichlet": (I, [P, P]), "afg_forest_get_solution": (I, [P, P]),
    "afg_forest_solve": (I, [P, P, P]), "afg_kernel_launches": (I, [P]),
    "afg_time_kernel": (I, [P, I, I, I, I, P, P, P, P]),
    "afg_forest_residual_norms_noalloc": (I, [P, P, P]),
    "afg_set_allocator": (I, [P, P, P]), "afg_cell_centers_device": (I, [P, P]),
    "afg_forest_time_kernel": (I, [P, I, I, I, I, P, P, P, P]),
    "afg_autotune": (I, [P, I, P, ctypes.c_char_p, P, ctypes.c_size_t]),
    "afg_set_operator": (I, [P, I]), "afg_set_eps": (I, [P, P]), "afg_forest_set_eps": (I, [P, P]),
    "afg_set_prolongation": (I, [P, I]), "afg_adapt_transfer": (I, [P, P, I, I, P, P]),
    "afg_flag_cells": (I, [P, P, I, DBL, DBL, P]),
}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEALLOC_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
# every callback pair ever installed: a buffer goes back to the callbacks that
# made it, so none of them may be freed while the process runs
_ALLOCATORS = []


def set_allocator(alloc, dealloc):
    """Route the library's device allocations through alloc(nbytes) -> int
    pointer and dealloc(pointer) (afg_set_allocator); both None restores
    cudaMalloc.  Set it before creating trees and forests."""
    if alloc is None and dealloc is None:
        _check(lib().afg_set_allocator(None, None, None))
        return

    def a(n, _ctx):
        try:
            return int(alloc(int(n)))
        except Exception:  # noqa: BLE001 - the library reports NULL as AFG_ERR_NOMEM
            return None

    def d(ptr, _ctx):
        dealloc(int(ptr))

    cbs = (ALLOC_FN(a), DEALLOC_FN(d))
    _ALLOCATORS.append(cbs)
    _check(lib().afg_set_allocator(ctypes.cast(cbs[0], P), ctypes.cast(cbs[1], P), None))


def use_torch_allocator():
    """Take the library's device memory from PyTorch's caching allocator (on
    the stream current at each allocation)."""
    import torch
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n), torch.cuda.caching_allocator_delete)


def kernel_launches():
    c = ctypes.c_ulonglong(0)
    _check(lib().afg_kernel_launches(ctypes.byref(c)))
    return c.value


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libafgpu (compiling it first if sources changed and nvcc exists)."""
    global _LIB
    if _LIB is None:
        if build_if_missing:
            try:
                _build.build()
            except RuntimeError:
                if not os.path.exists(_build.LIB):
                    raise
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libafgpu.so is not built (%s); run paper_1701_04329_gb300/build.py" % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, allow=()):
    if rc != AFG_OK and rc not in allow:
        raise AfgError(rc, lib().afg_last_error().decode())
    return rc


def default_opts(**kw):
    o = MgOpts()
    lib().afg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %s" % k)
        setattr(o, k, v)
    return o


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(P)


def _dev(t, n=None):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d values, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Tree:
    """A quadtree (dim=2) or octree (dim=3) on [0,1]^dim, root box of box_n^dim
    cells (Sec. 2.1-2.2), with its multigrid data on the GPU.  roots=(rx, ry[,
    rz]) makes level 1 a block of root boxes, the domain [0,rx] x [0,ry] (x
    [0,rz]) (not in forests)."""

    def __init__(self, dim, box_n, max_level, roots=None):
        self.D, self.N, self.max_level = dim, box_n, max_level
        h = ctypes.c_void_p()
        if roots is None:
            self.roots = (1,) * dim
            _check(lib().afg_tree_create(dim, box_n, max_level, ctypes.byref(h)))
        else:
            self.roots = tuple(int(r) for r in roots)
            if len(self.roots) != dim:
                raise ValueError("roots needs one count per axis")
            nr = (ctypes.c_int * dim)(*self.roots)
            _check(lib().afg_tree_create_roots(dim, box_n, max_level, nr, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.afg_tree_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ---- tree (host) ----------------------------------------------------------
    def refine_uniform(self, level):
        _check(lib().afg_refine_uniform(self._h, level))

    def info(self):
        i = TreeInfo()
        _check(lib().afg_info(self._h, ctypes.byref(i)))
        return i

    @property
    def n_leaf_cells(self):
        return self.info().n_leaf_cells

    @property
    def n_bfaces(self):
        return self.info().n_bfaces

    def cell_centers(self):
        x = np.zeros((self.n_leaf_cells, self.D))
        _check(lib().afg_cell_centers(self._h, x.ctypes.data_as(P)))
        return x

    def cell_centers_device(self, out=None):
        """Leaf cell centres as a (n_leaf_cells, dim) float64 CUDA tensor,
        written by the library's kernel."""
        import torch
        self._sync_stream()
        n = self.n_leaf_cells
        if out is None:
            out = torch.empty((n, self.D), dtype=torch.float64, device="cuda")
        _check(lib().afg_cell_centers_device(self._h, _dev(out.view(-1), n * self.D)))
        return out

    def face_centers(self):
        x = np.zeros((self.n_bfaces, self.D))
        _check(lib().afg_face_centers(self._h, x.ctypes.data_as(P)))
        return x

    def leaf_levels(self):
        out = np.zeros(self.info().n_leaves, np.int32)
        _check(lib().afg_leaf_levels(self._h, out.ctypes.data_as(P)))
        return out

    def adapt(self, flags, n_buf=2):
        f, fp = _np(flags, np.int8)
        if f.size != self.n_leaf_cells:
            raise ValueError("need one flag per leaf cell")
        a, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().afg_adapt(self._h, fp, n_buf, ctypes.byref(a), ctypes.byref(r)))
        return a.value, r.value

    def flag_cells(self, f, power=2, tau_refine=1e-3, tau_coarsen=-1.0):
        """afg_flag_cells: int8 CUDA tensor of refinement flags from the leaf
        field f (+1 where |f| h^power > tau_refine, -1 below tau_coarsen)."""
        import torch
        self._sync_stream()
        out = torch.empty(self.n_leaf_cells, dtype=torch.int8, device="cuda")
        _check(lib().afg_flag_cells(self._h, _dev(f, self.n_leaf_cells), int(power), float(tau_refine),
                                    float(tau_coarsen), ctypes.c_void_p(out.data_ptr())))
        return out

    def adapt_transfer(self, flags, n_buf=2, scheme=AFG_PROLONG_LINEAR):
        """afg_adapt_transfer: adapt and carry the device solution along."""
        f, fp = _np(flags, np.int8)
        if f.size != self.n_leaf_cells:
            raise ValueError("need one flag per leaf cell")
        self._sync_stream()
        a, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().afg_adapt_transfer(self._h, fp, n_buf, int(scheme), ctypes.byref(a), ctypes.byref(r)))
        return a.value, r.value

    def export(self):
        info = self.info()
        n, D = info.n_boxes, self.D
        level = np.zeros(n, np.int32)
        idx = np.zeros((n, D), np.int32)
        parent = np.zeros(n, np.int32)
        children = np.zeros((n, 2 ** D), np.int32)
        nbs = np.zeros((n, 3 ** D - 1), np.int32)
        _check(lib().afg_export_tree(self._h, *(a.ctypes.data_as(P) for a in (level, idx, parent, children, nbs))))
        return dict(level=level, idx=idx, parent=parent, children=children, neighbours=nbs)

    # ---- fields (device) -----------------------------------------------------
    def _sync_stream(self):
        _check(lib().afg_set_stream(self._h, _stream_ptr()))

    def set_rhs(self, rho):
        self._sync_stream()
        _check(lib().afg_set_rhs(self._h, _dev(rho, self.n_leaf_cells)))

    def set_dirichlet(self, b):
        self._sync_stream()
        _check(lib().afg_set_dirichlet(self._h, _dev(b, self.n_bfaces)))

    def set_boundary_types(self, types):
        """Per domain side (-x,+x,-y,+y[,-z,+z]): AFG_BC_DIRICHLET,
        AFG_BC_NEUMANN or AFG_BC_PERIODIC (pairs; set on the root box before
        refining).  Discards the device fields: set rho and b after it."""
        t = np.ascontiguousarray(types, dtype=np.int32)
        if t.size != 2 * self.D:
            raise ValueError("need %d boundary types" % (2 * self.D))
        _check(lib().afg_set_boundary_types(self._h, t.ctypes.data_as(P)))

    def set_operator(self, op):
        """AFG_OP_LAPLACE, AFG_OP_VAR (div(eps grad u), Sec. 3.4) or
        AFG_OP_VAR_RZ ((r,z) coordinates, Sec. 3.5); then set eps."""
        _check(lib().afg_set_operator(self._h, int(op)))

    def set_eps(self, eps):
        self._sync_stream()
        _check(lib().afg_set_eps(self._h, _dev(eps, self.n_leaf_cells)))

    def set_prolongation(self, scheme):
        """AFG_PROLONG_LINEAR (default), AFG_PROLONG_MULTILINEAR or
        AFG_PROLONG_ZEROTH for the coarse-grid correction (Sec. 2.5)."""
        _check(lib().afg_set_prolongation(self._h, int(scheme)))

    def set_solution(self, u):
        self._sync_stream()
        _check(lib().afg_set_solution(self._h, _dev(u, self.n_leaf_cells)))

    def get_solution(self, out=None):
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(self.n_leaf_cells, dtype=torch.float64, device="cuda")
        _check(lib().afg_get_solution(self._h, _dev(out, self.n_leaf_cells)))
        return out

    def fmg(self, opts=None):
        self._sync_stream()
        st = Stats()
        _check(lib().afg_fmg(self._h, ctypes.byref(opts or default_opts()), ctypes.byref(st)))
        return st.as_dict()

    def vcycle(self, opts=None):
        self._sync_stream()
        st = Stats()
        _check(lib().afg_vcycle(self._h, ctypes.byref(opts or default_opts()), ctypes.byref(st)))
        return st.as_dict()

    def solve(self, opts=None, allow_not_converged=False):
        self._sync_stream()
        st = Stats()
        allow = (AFG_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        _check(lib().afg_solve(self._h, ctypes.byref(opts or default_opts()), ctypes.byref(st)), allow)
        return st.as_dict()

    def residual_norm(self):
        self._sync_stream()
        r, p = ctypes.c_double(), ctypes.c_double()
        _check(lib().afg_residual_norm(self._h, ctypes.byref(r), ctypes.byref(p)))
        return r.value, p.value

    def time_kernel(self, kernel, level, fp64=True, reps=20):
        """Mean duration (ms) of one kernel launch plus its algorithmic bytes,
        flops and cells (see afg_time_kernel)."""
        self._sync_stream()
        ms, by, fl, nc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        _check(lib().afg_time_kernel(self._h, kernel, level, int(fp64), reps, ctypes.byref(ms), ctypes.byref(by),
                                     ctypes.byref(fl), ctypes.byref(nc)))
        return dict(ms=ms.value, bytes=by.value, flops=fl.value, cells=nc.value)

    def adjoint(self, g, opts=None):
        """Solve K^T lam = g; returns (lam = dL/drho, dL/db) as CUDA tensors."""
        import torch
        self._sync_stream()
        lam = torch.empty(self.n_leaf_cells, dtype=torch.float64, device="cuda")
        db = torch.empty(max(self.n_bfaces, 1), dtype=torch.float64, device="cuda")
        st = Stats()
        _check(lib().afg_adjoint(self._h, _dev(g, self.n_leaf_cells), _dev(lam), _dev(db),
                                 ctypes.byref(opts or default_opts()), ctypes.byref(st)))
        return lam, db[: self.n_bfaces], st.as_dict()


class Forest:
    """Independent trees solved together (per-level box lists concatenated)."""

    def __init__(self, trees):
        arr = (ctypes.c_void_p * len(trees))(*[t._h.value for t in trees])
        h = ctypes.c_void_p()
        _check(lib().afg_forest_create(len(trees), arr, ctypes.byref(h)))
        self._h = h
        self.T = len(trees)
        self.cells = np.zeros(self.T, np.int64)
        self.faces = np.zeros(self.T, np.int64)
        _check(lib().afg_forest_counts(self._h, self.cells.ctypes.data_as(P), self.faces.ctypes.data_as(P)))

    def close(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.afg_forest_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _sync_stream(self):
        _check(lib().afg_forest_set_stream(self._h, _stream_ptr()))

    def set_rhs(self, rho):
        self._sync_stream()
        _check(lib().afg_forest_set_rhs(self._h, _dev(rho, int(self.cells.sum()))))

    def set_dirichlet(self, b):
        self._sync_stream()
        _check(lib().afg_forest_set_dirichlet(self._h, _dev(b, int(self.faces.sum()))))

    def set_eps(self, eps):
        self._sync_stream()
        _check(lib().afg_forest_set_eps(self._h, _dev(eps, int(self.cells.sum()))))

    def get_solution(self, out=None):
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(int(self.cells.sum()), dtype=torch.float64, device="cuda")
        _check(lib().afg_forest_get_solution(self._h, _dev(out, int(self.cells.sum()))))
        return out

    def residual_norms_noalloc(self):
        """Per-tree (max|r|, max|rho|) through the allocation-free entry point."""
        self._sync_stream()
        r = np.zeros(self.T)
        p = np.zeros(self.T)
        _check(lib().afg_forest_residual_norms_noalloc(self._h, r.ctypes.data_as(P), p.ctypes.data_as(P)))
        return r, p

    def time_kernel(self, kernel, level, fp64=True, reps=20):
        """afg_forest_time_kernel: mean ms of one launch over the level's boxes
        of every tree, with its algorithmic bytes, flops and cells."""
        self._sync_stream()
        ms, by, fl, nc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        _check(lib().afg_forest_time_kernel(self._h, kernel, level, int(fp64), reps, ctypes.byref(ms),
                                            ctypes.byref(by), ctypes.byref(fl), ctypes.byref(nc)))
        return dict(ms=ms.value, bytes=by.value, flops=fl.value, cells=nc.value)

    def solve(self, opts=None, allow_not_converged=False):
        self._sync_stream()
        st = (Stats * self.T)()
        allow = (AFG_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        _check(lib().afg_forest_solve(self._h, ctypes.byref(opts or default_opts()), st), allow)
        return [s.as_dict() for s in st]
