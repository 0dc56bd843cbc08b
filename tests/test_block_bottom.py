"""The coarse levels of a block of root boxes as rectangular grids
(csrc/block_bottom.cuh, built here for the host and run with one thread)
against the oracle's box-by-box cycle on a tree made of the root boxes alone
(arXiv:1701.04329 Sec. 2.2 and 3.2: a non-square domain has several boxes
on the coarse grids; reading 22).  On such a tree the oracle's V-cycle and
FMG cycle are exactly the part of the cycle at and below level 1, so the
two must agree bit for bit: same ghost rules, same sums in the same order.
No GPU."""
import os
import subprocess

import numpy as np
import pytest

from oracle.oracle import OracleTree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("blk")
    exe = str(d / "block_bottom_host")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(ROOT, "tests", "block_bottom_host.cpp")], check=True)
    return exe, d


def rect_index(x, h, n):
    q = np.floor(x / h).astype(np.int64)
    lin = q[:, 0]
    mul = n[0]
    for a in range(1, x.shape[1]):
        lin = lin + mul * q[:, a]
        mul *= n[a]
    return lin


def run(harness, D, N, roots, types, mode, seed, nd=2, nu=2, nb=4, op=0):
    exe, d = harness
    t = OracleTree(D, N, 1, roots=roots)
    bct = list(types) if types is not None else [0] * (2 * D)
    if types is not None:
        t.set_boundary_types(types)
    rng = np.random.default_rng(seed)
    eps = np.exp(rng.normal(size=t.n_leaf_cells)) if op else np.ones(t.n_leaf_cells)
    if op:
        t.set_operator(op)
        t.set_eps(eps)
    rho = rng.normal(size=t.n_leaf_cells)
    b = rng.normal(size=t.n_bfaces)
    u0 = 0.1 * rng.normal(size=t.n_leaf_cells)
    t.set_rhs(rho)
    t.set_dirichlet(b)
    t.set_solution(u0)
    (t.vcycle if mode == 0 else t.fmg)(nd, nu, nb)
    uo = t.get_solution()
    # the same data in rectangle order
    h = 1.0 / N
    n = [r * N for r in roots]
    lin = rect_index(t.cell_centers(), h, n)
    rrho = np.zeros(t.n_leaf_cells)
    ru0 = np.zeros(t.n_leaf_cells)
    rrho[lin], ru0[lin] = rho, u0
    reps = np.zeros(t.n_leaf_cells)
    reps[lin] = eps
    fc = t.face_centers()
    faces = []
    for s in range(2 * D):
        if bct[s] == 2:
            continue
        a, hi = s // 2, s % 2
        on = fc[:, a] == (roots[a] if hi else 0.0)
        t1 = 1 if a == 0 else 0
        t2 = (1 if a == 2 else 2) if D == 3 else None
        f = np.floor(fc[on, t1] / h).astype(np.int64)
        if t2 is not None:
            f = f + n[t1] * np.floor(fc[on, t2] / h).astype(np.int64)
        arr = np.zeros(int(on.sum()))
        arr[f] = b[on]
        faces.append(arr)
    hdr = np.array([D, N] + list(roots) + [1] * (3 - D) + bct + [0] * (6 - 2 * D) + [mode, nd, nu, nb, op], np.int32)
    fin, fout = str(d / "in.bin"), str(d / "out.bin")
    with open(fin, "wb") as f:
        f.write(hdr.tobytes())
        f.write(rrho.tobytes())
        f.write(ru0.tobytes())
        f.write(reps.tobytes())
        for arr in faces:
            f.write(arr.tobytes())
    subprocess.run([exe, fin, fout], check=True)
    ub = np.fromfile(fout, np.float64)
    assert np.abs(uo - u0).max() > 1e-3  # the cycle did change the solution
    return uo, ub[lin]


CASES = [(2, 8, (2, 1), None), (2, 8, (3, 2), [0, 1, 0, 0]), (2, 16, (1, 3), [2, 2, 0, 0]),
         (2, 4, (4, 1), [0, 0, 2, 2]), (3, 8, (2, 1, 1), None), (3, 4, (1, 2, 2), [0, 1, 2, 2, 0, 0]),
         (3, 8, (2, 2, 1), [2, 2, 0, 0, 1, 0])]


@pytest.mark.parametrize("D,N,roots,types", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_block_grids_match_the_oracle_bit_for_bit(harness, D, N, roots, types, mode):
    uo, ub = run(harness, D, N, roots, types, mode, seed=7 + N + len(roots) + mode)
    assert np.array_equal(uo, ub), np.abs(uo - ub).max()


def test_other_smoothing_counts(harness):
    uo, ub = run(harness, 2, 8, (3, 1), [0, 1, 0, 0], 0, seed=3, nd=1, nu=3, nb=6)
    assert np.array_equal(uo, ub)


@pytest.mark.parametrize("D,N,roots,types,op", [(2, 8, (2, 1), None, 1), (2, 8, (3, 2), [0, 1, 2, 2], 1),
                                                (3, 4, (2, 1, 1), [0, 0, 0, 1, 2, 2], 1), (2, 8, (2, 1), None, 2),
                                                (2, 16, (1, 2), [0, 0, 0, 1], 2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_variable_coefficient_block_grids_match_the_oracle(harness, D, N, roots, types, op, mode):
    """div(eps grad u) with a random positive eps per cell, and its (r,z)
    form (volume-weighted restriction, radii from each root's origin)."""
    uo, ub = run(harness, D, N, roots, types, mode, seed=31 + N + op + mode, op=op)
    assert np.array_equal(uo, ub), np.abs(uo - ub).max()
