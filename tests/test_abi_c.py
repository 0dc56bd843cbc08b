"""The C ABI from plain C: tests/abi_tree_example.c (tree calls, no GPU) and
tests/abi_solve_example.c (a whole solve on the GPU with a counting
allocator) are compiled with gcc -std=c11 -pedantic against include/afgpu.h,
linked with libafgpu.so, run, and their figures compared with the oracle."""
import os
import subprocess

import numpy as np
import pytest

from oracle.oracle import OracleTree
from paper_1701_04329_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tree_calls_from_c(tmp_path):
    lib = B.build()
    exe = str(tmp_path / "abi_tree_example")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_tree_example.c"), "-o", exe, "-L", os.path.dirname(lib),
                    "-lafgpu", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    rows = {l.split()[0]: l.split()[1:] for l in out}
    a = OracleTree(2, 8, 5)
    a.refine_uniform(3)
    assert rows["uniform"] == [str(a.nbox), str(a.n_leaf_cells), str(a.n_bfaces)]
    flags = np.zeros(a.n_leaf_cells, np.int8)
    flags[0] = 1
    added, removed = a.adapt(flags, 2)
    assert rows["adapted"] == [str(added), str(removed), str(a.nbox), str(a.n_leaf_cells), str(a.n_bfaces)]
    e = a.export()
    assert rows["export"] == [str(e["level"][0]), str(e["parent"][0]), str(e["level"].max())]
    assert rows["error"][0] == "1" and "dim" in " ".join(rows["error"][1:])
    m = OracleTree(2, 8, 3, roots=(3, 2))
    m.refine_uniform(2)
    assert rows["roots"] == [str(m.nbox), str(m.n_leaf_cells), str(m.n_bfaces)]


@pytest.mark.gpu
def test_solve_from_c_with_a_counting_allocator(tmp_path):
    """A whole solve from plain C (tests/abi_solve_example.c): the library's
    device buffers come from the program's allocator callbacks, which see
    every allocation returned by the time the tree is destroyed; the
    solution matches the FP64 oracle's after the same number of cycles."""
    lib = B.build()
    exe = str(tmp_path / "abi_solve_example")
    cuda = "/usr/local/cuda"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "abi_solve_example.c"), "-o", exe,
                    "-L", os.path.dirname(lib), "-lafgpu", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-Wl,-rpath," + os.path.dirname(lib) + ":" + os.path.join(cuda, "lib64")], check=True)
    sol = str(tmp_path / "u.bin")
    out = subprocess.run([exe, sol], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    rows = {l.split()[0]: l.split()[1:] for l in out.stdout.splitlines()}
    allocs_during, allocs, frees, live = (int(v) for v in rows["allocator"])
    assert allocs_during > 0 and allocs == allocs_during == frees and live == 0
    a = OracleTree(2, 8, 5)
    a.refine_uniform(4)
    x = a.cell_centers()
    a.set_rhs(x[:, 0] * (1.0 - x[:, 0]) - x[:, 1])
    a.set_dirichlet(np.zeros(a.n_bfaces))
    a.zero_solution()
    cycles = a.solve(1e-10, 50)
    assert int(rows["solve"][0]) == cycles
    u = np.fromfile(sol, dtype=np.float64)
    ref = a.get_solution()
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()
