"""The forest autotuner: every candidate converges, the choice is the fastest
converged candidate, and box sizes 8 and 16 give the same finest spacing."""
import pytest

from paper_1701_04329_gb300 import afgpu, autotune

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotuner_picks_fastest_converged_configuration():
    best, table = autotune.autotune_forest(n_trees=8, reps=1, max_level_cap=6, sweeps=((1, 1), (2, 2)))
    assert len(table) == 4
    assert all(r["converged"] for r in table)
    assert best["ms"] == min(r["ms"] for r in table)
    assert {r["box_n"] for r in table} == {8, 16}
    # same finest spacing: the 16^2-box forest has as many leaf cells near the sources
    cells = {r["box_n"]: r["unknowns"] for r in table}
    assert 0.5 < cells[16] / cells[8] < 4.0
