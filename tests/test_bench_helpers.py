"""Host helpers of bench.py: the roofline denominator, the traffic figure's
validity rule, and the whole-job rate."""

import json
import os

import pytest

import bench


def test_peak_is_the_measured_copy_rate_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6788.6, "bf16_tflops": 1911.4}))
    assert bench.measured_peaks() == (6788.6, "measured")


def test_traffic_holds_only_for_the_captured_sources(tmp_path, monkeypatch):
    root = tmp_path
    csrc = root / "paper_2112_09972_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.ROW_KERNEL_SOURCES:
        (csrc / name).write_text(f"// {name}\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.row_kernel_sha1()
    (root / "profiles").mkdir()
    (root / "profiles" / "traffic.json").write_text(json.dumps(
        {"box128": {"dram_bytes_per_launch": 652582656, "source_sha1": sha}}))
    assert bench.kernel_traffic("box128") == 652582656
    assert bench.kernel_traffic("other") is None
    (csrc / bench.ROW_KERNEL_SOURCES[0]).write_text("// changed\n")  # a kernel edit voids the figure
    assert bench.row_kernel_sha1() != sha
    assert bench.kernel_traffic("box128") is None


def test_committed_traffic_entries_are_consistent():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles", "traffic.json")
    with open(path) as fh:
        d = json.load(fh)
    for key, e in d.items():
        total = e["dram_read_bytes"] + e["dram_write_bytes"]
        assert e["dram_bytes_per_launch"] == total, key
        # DRAM bytes of a launch are within a few per cent of its
        # algorithmic bytes when nothing is re-read; a little below them
        # when some reads hit lines the previous launch left in L2 (the
        # ghost values the ghost kernel writes just before)
        assert 0.95 <= total / e["algorithmic_bytes_per_launch"] < 1.1, key


def test_job_rate_counts_every_rank():
    assert bench.job_rate(2_097_152, 100, 1, 0.02) == pytest.approx(10_485.76)
    assert bench.job_rate(2_097_152, 100, 4, 0.02) == pytest.approx(4 * 10_485.76)
