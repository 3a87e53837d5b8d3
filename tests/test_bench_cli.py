"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the one-JSON-line contract for every scheme the command line selects; run
on the small hexagon workload so it takes seconds."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def run(*extra):
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                          "--workload", "hex_1024", "--steps", "2", "--warmup", "1", *extra],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("extra,scheme", [((), "LTS3"), (("--order", "2", "--dt-scale", "0.5"), "LTS2"),
                                          (("--interface-layers", "2"), "LTS3 with 2-cell interfaces")])
def test_reference_arm_line(extra, scheme):
    line = run(*extra)
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert f"{scheme} M=2" in line["config"]["workload"]
    assert "doubly periodic hexagons" in line["config"]["workload"]


def test_dt_scale_is_reported():
    a = run()
    b = run("--dt-scale", "0.5")
    assert abs(b["config"]["dt_coarse_s"] - 0.5 * a["config"]["dt_coarse_s"]) <= 1e-12 * a["config"]["dt_coarse_s"]
