"""The C-ABI library loads without a GPU and exports every symbol that
include/afgpu.h declares (no compute calls)."""
import ctypes
import os
import re

from paper_1701_04329_gb300 import afgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "afgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = afgpu.lib()
    names = declared_symbols()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
        assert n in afgpu._SIGS, n


def test_errors_are_status_codes():
    L = afgpu.lib()
    h = ctypes.c_void_p()
    assert L.afg_tree_create(4, 8, 3, ctypes.byref(h)) == afgpu.AFG_ERR_ARG
    assert b"dim" in L.afg_last_error()
    assert L.afg_tree_create(2, 6, 3, ctypes.byref(h)) == afgpu.AFG_ERR_ARG
    assert L.afg_tree_create(3, 8, 22, ctypes.byref(h)) == afgpu.AFG_ERR_ARG
    bad = (ctypes.c_int * 3)(2, 0, 1)
    assert L.afg_tree_create_roots(3, 8, 4, bad, ctypes.byref(h)) == afgpu.AFG_ERR_ARG
    big = (ctypes.c_int * 2)(64, 1)
    assert L.afg_tree_create_roots(2, 8, 17, big, ctypes.byref(h)) == afgpu.AFG_ERR_ARG  # 64 << 16 > 2^21
    assert b"Morton" in L.afg_last_error()
    # a block of root boxes: the tree calls work without a GPU
    m = afgpu.Tree(2, 8, 4, roots=(2, 1))
    m.refine_uniform(2)
    assert m.n_leaf_cells == 2 * 4 * 64
    t = afgpu.Tree(2, 8, 4)
    try:
        t.refine_uniform(9)
        assert False, "expected an error"
    except afgpu.AfgError as e:
        assert e.code == afgpu.AFG_ERR_ARG
    import numpy as np
    try:
        t.adapt(np.full(t.n_leaf_cells, 3, np.int8))
        assert False
    except afgpu.AfgError as e:
        assert e.code == afgpu.AFG_ERR_ARG
    try:
        t.adapt(np.zeros(t.n_leaf_cells, np.int8), n_buf=9)
        assert False
    except afgpu.AfgError as e:
        assert e.code == afgpu.AFG_ERR_ARG
    assert t.info().n_boxes == 1  # failed calls left the tree unchanged


def test_boundary_types_validated_on_the_host():
    """afg_set_boundary_types: 0/1/2 per side, periodic sides in pairs; a
    refused call leaves the types (and the tree) unchanged.  Only Neumann
    sides (a singular problem) are accepted."""
    import numpy as np
    t = afgpu.Tree(2, 8, 4)
    t.refine_uniform(2)
    for bad in ([0, 2, 0, 0], [0, -1, 0, 0], [3, 0, 0, 0]):
        try:
            t.set_boundary_types(bad)
            assert False, bad
        except afgpu.AfgError as e:
            assert e.code == afgpu.AFG_ERR_ARG
    t.set_boundary_types([afgpu.AFG_BC_NEUMANN, afgpu.AFG_BC_DIRICHLET, afgpu.AFG_BC_NEUMANN, afgpu.AFG_BC_DIRICHLET])
    assert t.info().n_boxes == 5
    t.set_boundary_types([afgpu.AFG_BC_NEUMANN] * 4)
    t.set_operator(afgpu.AFG_OP_LAPLACE)
    try:  # the variable-coefficient operators need a Dirichlet side
        t.set_operator(afgpu.AFG_OP_VAR)
        assert False
    except afgpu.AfgError as e:
        assert e.code == afgpu.AFG_ERR_ARG
    try:
        t.set_boundary_types([1, 0, 1])  # wrong count for 2D
        assert False
    except ValueError:
        pass


def test_periodic_types_validated_on_the_host():
    """Periodic sides come in pairs and switch only on the root box alone."""
    t = afgpu.Tree(3, 8, 4)
    for bad in ([2, 0, 0, 0, 0, 0], [2, 1, 0, 0, 0, 0], [0, 0, 0, 0, 1, 2]):
        try:
            t.set_boundary_types(bad)
            assert False, bad
        except afgpu.AfgError as e:
            assert e.code == afgpu.AFG_ERR_ARG
    t.set_boundary_types([afgpu.AFG_BC_PERIODIC] * 2 + [afgpu.AFG_BC_DIRICHLET] * 4)
    t.refine_uniform(2)
    try:
        t.set_boundary_types([0] * 6)
        assert False
    except afgpu.AfgError as e:
        assert e.code == afgpu.AFG_ERR_ARG
    t.set_boundary_types([2, 2, 1, 0, 0, 0])  # Neumann/Dirichlet changes stay allowed
    assert t.n_bfaces == 4 * 4 * 64  # no boundary faces on the periodic x sides


def test_allocator_needs_both_callbacks():
    """afg_set_allocator: both callbacks or neither (no GPU involved)."""
    L = afgpu.lib()
    f = afgpu.ALLOC_FN(lambda n, c: None)
    assert L.afg_set_allocator(ctypes.cast(f, ctypes.c_void_p), None, None) == afgpu.AFG_ERR_ARG
    assert b"both" in L.afg_last_error()
    assert L.afg_set_allocator(None, None, None) == afgpu.AFG_OK


def test_operator_validated_on_the_host():
    """afg_set_operator: known operators only, (r,z) in 2D only; a tree of
    several root boxes takes it before its data; eps needs a
    variable-coefficient operator first (no GPU needed)."""
    t = afgpu.Tree(3, 8, 2)
    for bad in (3, -1, afgpu.AFG_OP_VAR_RZ):
        try:
            t.set_operator(bad)
            assert False, bad
        except afgpu.AfgError as e:
            assert e.code == afgpu.AFG_ERR_ARG
    m = afgpu.Tree(2, 8, 2, roots=(2, 1))
    m.set_operator(afgpu.AFG_OP_VAR)  # no data yet: the coarse grids go to the per-level kernels
    m.set_prolongation(afgpu.AFG_PROLONG_MULTILINEAR)
    L = afgpu.lib()
    assert L.afg_set_eps(t._h, ctypes.c_void_p(8)) == afgpu.AFG_ERR_STATE
    afgpu.Tree(2, 8, 2).set_operator(afgpu.AFG_OP_VAR_RZ)
