"""The forest autotuner (afg_autotune, called from Python): every candidate
converges, the choice is the converged candidate with the most unknowns per
second, box sizes 8 and 16 give the same finest spacing, both threads-per-box
choices of the FP32 half-sweep are tried, and a malformed search space is
refused."""
import ctypes

import pytest

from paper_1701_04329_gb300 import afgpu, autotune

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotuner_picks_most_unknowns_per_second():
    best, table = autotune.autotune_forest(n_trees=8, reps=1, max_level_cap=6, sweeps=((1, 1), (2, 2)))
    assert len(table) == 8  # 2 box sizes x 2 sweep pairs x 2 threads-per-box choices
    assert {r["threads_per_box"] for r in table} == {4, 8, 16, 32}  # 8^2 boxes: 8 or 4; 16^2: 32 or 16
    assert all(r["converged"] for r in table)
    assert best["unknowns_per_s"] == max(r["unknowns_per_s"] for r in table)
    for r in table:
        assert abs(r["unknowns_per_s"] - r["unknowns"] / (r["ms"] * 1e-3)) <= 1e-5 * r["unknowns_per_s"]
    assert {r["box_n"] for r in table} == {8, 16}
    # same finest spacing: the 16^2-box forest has as many leaf cells near the sources
    cells = {r["box_n"]: r["unknowns"] for r in table}
    assert 0.5 < cells[16] / cells[8] < 4.0


def test_autotune_rejects_a_malformed_search_space():
    trees, rho, b = autotune.build_forest(2, 8, max_level_cap=5)
    f = afgpu.Forest(trees)
    f.set_rhs(torch.tensor(rho, device="cuda"))
    arr = (ctypes.c_void_p * 1)(f._h.value)
    out = ctypes.create_string_buffer(4096)
    for bad in (b'{"sweeps": [[1, 1], [2]]}', b'{"reps": 0}', b'{"sweeps": [[1, x]]}', b'{"vectors_per_thread": [3]}'):
        rc = afgpu.lib().afg_autotune(arr, 1, None, bad, out, len(out))
        assert rc == afgpu.AFG_ERR_ARG, bad
    small = ctypes.create_string_buffer(16)
    rc = afgpu.lib().afg_autotune(arr, 1, None, b'{"sweeps": [[1, 1]], "reps": 1}', small, len(small))
    assert rc == afgpu.AFG_ERR_ARG and b"too small" in afgpu.lib().afg_last_error()
