"""The work-count model of the LTS speed-up that bench.py reports beside the
measured one, pinned to the paper's printed example (Section 3.3, Table 3):
with the interface cells counted among the coarse time-step cells and no
extra first-stage cells, as the paper's definition does, the model reduces
to M N / (N_coarse-dt + M N_fine) and must give the printed 2.342."""
import json
from pathlib import Path

import numpy as np

import bench

GOLDEN = Path(__file__).resolve().parent / "golden" / "optimal_ratio_section3_3.json"


def counts(fine=0, fbar=0, interface=0, coarse=0):
    """Band counts in library order: F deep, F3, F2, F1, I1, I2, C1..C5, C rest."""
    c = np.zeros(12, np.int64)
    c[0] = fine - fbar
    c[2] = fbar
    c[4] = interface
    c[6] = coarse
    return c


def test_paper_optimal_ratio():
    g = json.loads(GOLDEN.read_text())
    assert g["coarse_cells"] + g["interface_cells"] == g["coarse_time_step_cells"]
    p = bench.predicted_speedup(counts(fine=g["fine_time_step_cells"], coarse=g["coarse_time_step_cells"]),
                                g["M"])
    assert round(p["predicted"], g["printed_digits"]) == g["optimal_ratio"]
    assert p["cells"]["fine"] + p["cells"]["coarse"] == 621007


def test_model_limits():
    # all cells coarse: every cell takes the coarse step, a gain of M; all
    # cells fine: no gain
    assert bench.predicted_speedup(counts(coarse=1000), 8)["predicted"] == 8.0
    assert bench.predicted_speedup(counts(fine=1000), 8)["predicted"] == 1.0
    # LTS3 interface cells cost 2 + 3M evaluations, the extra first-stage
    # fine cells one more each: both lower the gain
    base = bench.predicted_speedup(counts(fine=100, coarse=900), 4)["predicted"]
    assert bench.predicted_speedup(counts(fine=100, interface=20, coarse=880), 4)["predicted"] < base
    assert bench.predicted_speedup(counts(fine=100, fbar=10, coarse=900), 4)["predicted"] < base
