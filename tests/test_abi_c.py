"""The C ABI from plain C (no Python, no GPU): tests/abi_tree_example.c is
compiled with gcc -std=c11 -pedantic against include/afgpu.h, linked with
libafgpu.so, run, and its figures compared with the oracle's tree."""
import os
import subprocess

import numpy as np

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
