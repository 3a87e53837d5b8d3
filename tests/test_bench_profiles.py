"""bench.py reads the committed ncu summaries only while they describe the
kernels that are built: the DRAM traffic per ring launch and the device-time
shares carry the hash of kernels.cu they were captured with."""
import bench


def test_profiles_parse_and_match_the_kernels():
    h = bench.kernel_hash()
    assert len(h) == 16
    traffic = bench.dram_traffic_per_launch()
    shares = bench.device_time_shares()
    # the committed summaries are kept in step with kernels.cu
    assert traffic is not None and traffic > 1e6
    assert shares is not None and set(shares) == {"vertex", "ring", "edge"}
    assert abs(sum(shares.values()) - 1.0) < 1e-3


def test_profiles_ignored_for_other_kernels(monkeypatch):
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0000000000000000")
    assert bench.dram_traffic_per_launch() is None
    assert bench.device_time_shares() is None
