"""bench.py reads the committed ncu summaries only while they describe the
kernels that are built: the DRAM traffic per ring launch and the device-time
shares carry the hash of kernels.cu's code (comments and blank lines
removed) they were captured with."""
import json
import re

import bench


def block(path):
    m = re.search(r"```json\s*(\{.*?\})\s*```", path.read_text(), re.S)
    assert m, path
    return json.loads(m.group(1))


def test_summaries_carry_a_hash_and_their_figures():
    t = block(bench.TRAFFIC_SUMMARY)
    s = block(bench.LAUNCH_SUMMARY)
    assert len(t["kernels_cu_code_sha256_16"]) == 16 and t["ring_dram_bytes_per_launch"] > 1e6
    assert len(s["kernels_cu_code_sha256_16"]) == 16 and set(s["shares"]) == {"vertex", "ring", "edge"}
    assert abs(sum(s["shares"].values()) - 1.0) < 1e-3


def test_figures_used_only_for_the_kernels_they_describe(monkeypatch):
    t = block(bench.TRAFFIC_SUMMARY)
    monkeypatch.setattr(bench, "kernel_hash", lambda: t["kernels_cu_code_sha256_16"])
    assert bench.dram_traffic_per_launch() == float(t["ring_dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0000000000000000")
    assert bench.dram_traffic_per_launch() is None
    assert bench.device_time_shares() is None


def test_code_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    f = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "KERNEL_SRC", f)
    f.write_text("int a = 1;  // one\n/* a block\n   comment */\nint b = 2;\n")
    h0 = bench.kernel_hash()
    f.write_text("// reworded\nint a = 1;\n\n\nint b = 2;   /* other */\n")
    assert bench.kernel_hash() == h0
    f.write_text("int a = 1;\nint b = 3;\n")
    assert bench.kernel_hash() != h0
