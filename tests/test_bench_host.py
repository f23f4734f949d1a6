"""Host-side logic of bench.py (no GPU): the profile lookup that feeds the
roofline's `traffic`, the FP64 ALU roofline, the peak lookup."""
import json

import pytest

import bench


def test_profiled_figures_follow_the_kernel_source_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"dram_bytes_per_launch": 123, "fp64_inst_per_node": 83.0, "fp64_flop_per_node": 112.0}
    h = bench.kernel_source_hash()
    (prof / "step_kernel_traffic.json").write_text(json.dumps(
        {"kernel_source_hash": h, "workloads": {"rD2Q9-f64": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profiled_traffic("rD2Q9-f64") == 123
    assert bench.profiled_traffic("unknown") is None
    roof = bench.fp64_alu_roof("rD2Q9-f64", 8388608, 1.31958)
    # 83 pipe instructions per node at 8,388,608 nodes per 1.31958 ms
    assert roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(83.0 * 8388608 / 1.31958e-3 / 1e9, rel=1e-3)
    assert roof["frac"] == pytest.approx(roof["achieved"] / bench.FP64_PIPE_GINST, rel=1e-3)
    # counters taken on other kernel sources are not reported
    (prof / "step_kernel_traffic.json").write_text(json.dumps(
        {"kernel_source_hash": "0" * 16, "workloads": {"rD2Q9-f64": entry}}))
    assert bench.profiled_traffic("rD2Q9-f64") is None
    assert bench.fp64_alu_roof("rD2Q9-f64", 8388608, 1.3) is None


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.1}))
    assert bench.hbm_peak() == (6783.1, "measured")


def test_committed_profile_is_for_the_committed_kernels():
    """The committed ncu summary carries the hash of the step-kernel sources
    it was taken on; bench.py reports its traffic only while they match."""
    d = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "step_kernel_traffic.json")))
    assert len(d["kernel_source_hash"]) == 16
    assert "rD2Q9-f32" in d["workloads"]
    assert bench.host_cores() >= 1
