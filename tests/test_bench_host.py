"""Host-side helpers of bench.py (no GPU): the measured peak, and the DRAM
traffic taken from the committed ncu capture only while the kernel source it
was measured on is unchanged."""
import json
import os

import bench


def test_committed_traffic_follows_kernel_source():
    """Traffic is reported from the capture while its source hash is the current
    one (read + write bytes per launch), and never for another source."""
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        assert bench.committed_traffic("k_update") is None and bench.committed_traffic("k_deliver") is None
        return
    with open(path) as f:
        t = json.load(f)
    current = t["kernel_source_sha256_16"] == bench.kernel_source_hash()
    for k in ("k_update", "k_deliver"):
        v = bench.committed_traffic(k)
        if not current:
            assert v is None
            continue
        k_ = t["kernels"][k]
        assert v == k_["dram_bytes_per_launch"]
        assert abs(k_["dram_read_bytes_per_launch"] + k_["dram_write_bytes_per_launch"] - v) <= 1000.0
    assert bench.committed_traffic("k_unknown") is None


def test_stale_capture_reports_no_traffic(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.committed_traffic("k_update") is None


def test_measured_peak_is_read():
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) as f:
            assert kind == "measured" and peak == float(json.load(f)["hbm_gbs"])
    else:
        assert kind == "fallback"
