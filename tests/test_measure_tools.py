"""The ncu summary parsers behind profiles/ (CPU): launch shares with unit
scaling, and the DRAM-traffic record scaled to a full launch and tagged
with the kernels' source hash (which the bench checks before reporting it)."""
import csv
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

HEADER = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
          "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
          "Metric Unit", "Metric Value"]


def _write(path, rows, preamble=True):
    with open(path, "w", newline="") as f:
        if preamble:  # ncu prints its own log lines before the table
            f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HEADER)
        for k, (name, metric, unit, value) in enumerate(rows):
            w.writerow([k, 1, "python", "h", name, 1, 7, "(256, 1, 1)", "(152, 1, 1)", 0, "10.3",
                        "Command line profiler metrics", metric, unit, value])


def test_launch_summary_shares_and_units(tmp_path):
    from paper_1710_03608_gb300 import measure
    p = tmp_path / "launches.csv"
    _write(p, [
        ("void ctd::k_fiber_norms(const int *, int)", "gpu__time_duration.sum", "usecond", "250"),
        ("void ctd::k_fiber_norms(const int *, int)", "gpu__time_duration.sum", "nsecond",
         "250,000"),
        ("ctd::<unnamed>::k_cf<float, 4, 1>(ctd::CscDev)", "gpu__time_duration.sum", "msecond",
         "1.5"),
    ])
    out = measure.ncu_launch_summary(str(p)).splitlines()
    assert out[1].split()[0] == "ctd::<unnamed>::k_cf<float,"   # largest first
    norms = next(ln for ln in out if ln.startswith("ctd::k_fiber_norms"))
    f = norms.split()
    assert f[1] == "2" and float(f[2]) == pytest.approx(0.5) and f[3] == "25.00%"
    assert out[-1] == "total: 3 launches, 2.000 ms"


def test_traffic_record_scales_and_hashes(tmp_path):
    from paper_1710_03608_gb300 import measure
    src = tmp_path / "kernels.cu"
    src.write_text("__global__ void k_cf() {}\n")
    p = tmp_path / "traffic.csv"
    _write(p, [
        ("void ctd::k_copy_flat<float>(int)", "dram__bytes_read.sum", "Mbyte", "100"),
        ("void ctd::k_copy_flat<float>(int)", "dram__bytes_write.sum", "Gbyte", "0.2"),
        ("void ctd::k_cf<float, 4, 1>(int)", "dram__bytes_read.sum", "byte", "1,000,000"),
        ("void ctd::k_cf<float, 4, 1>(int)", "gpu__time_duration.sum", "usecond", "9"),
        ("void ctd::k_fiber_norms(int)", "dram__bytes_read.sum", "Mbyte", "999"),
    ])
    rec = measure.ncu_traffic_record(str(p), "k_copy_flat|k_cf", 2.5, str(src))
    assert rec["captured_bytes"] == pytest.approx(301e6)
    assert rec["bytes_per_launch"] == pytest.approx(2.5 * 301e6)
    assert rec["per_kernel_captured"] == {"ctd::k_copy_flat<float>": pytest.approx(300e6),
                                          "ctd::k_cf<float, 4, 1>": pytest.approx(1e6)}
    assert rec["source_sha"] == hashlib.sha256(src.read_bytes()).hexdigest()[:16]


def test_bench_reports_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    import json

    import bench
    src = tmp_path / "kernels.cu"
    src.write_text("A\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = hashlib.sha256(b"A\n").hexdigest()[:16]
    (prof / "traffic.json").write_text(json.dumps({"source_sha": sha, "bytes_per_launch": 5.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic(str(src))["bytes_per_launch"] == 5.0
    src.write_text("B\n")                    # the kernels changed since the capture
    assert bench.ncu_traffic(str(src)) is None


def test_dram_summary_groups_metrics_by_launch(tmp_path):
    """Three metrics per launch (read, write, duration) grouped by the launch
    ID: per kernel the mean duration, mean bytes and their rate."""
    from paper_1710_03608_gb300 import measure
    p = tmp_path / "dram.csv"
    rows = [
        (0, "void ctd::k_a(int)", "dram__bytes_read.sum", "Mbyte", "60"),
        (0, "void ctd::k_a(int)", "dram__bytes_write.sum", "Mbyte", "40"),
        (0, "void ctd::k_a(int)", "gpu__time_duration.sum", "usecond", "50"),
        (1, "void ctd::k_a(int)", "dram__bytes_read.sum", "byte", "100000000"),
        (1, "void ctd::k_a(int)", "dram__bytes_write.sum", "byte", "100000000"),
        (1, "void ctd::k_a(int)", "gpu__time_duration.sum", "nsecond", "150000"),
        (2, "ctd::k_b(int)", "dram__bytes_read.sum", "Kbyte", "1000"),
        (2, "ctd::k_b(int)", "dram__bytes_write.sum", "byte", "0"),
        (2, "ctd::k_b(int)", "gpu__time_duration.sum", "usecond", "10"),
    ]
    with open(p, "w", newline="") as f:
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HEADER)
        for lid, name, metric, unit, value in rows:
            w.writerow([lid, 1, "python", "h", name, 1, 7, "(256, 1, 1)", "(152, 1, 1)", 0,
                        "10.3", "Command line profiler metrics", metric, unit, value])
    out = measure.ncu_dram_summary(str(p), peak_gbs=1000.0).splitlines()
    a = out[1].split()
    # k_a: 2 launches, 100 us mean, 150 MB mean, 300 MB / 200 us = 1500 GB/s
    assert a[0] == "ctd::k_a" and a[1] == "2"
    assert float(a[2]) == pytest.approx(100.0) and float(a[3]) == pytest.approx(150.0)
    assert float(a[4]) == pytest.approx(1500.0) and float(a[5]) == pytest.approx(1.5)
    b = out[2].split()
    assert b[0] == "ctd::k_b" and float(b[4]) == pytest.approx(100.0)


def test_launch_summary_counts_only_durations(tmp_path):
    """On a capture with DRAM metrics beside the duration, the launch list
    sums the durations alone."""
    from paper_1710_03608_gb300 import measure
    p = tmp_path / "mixed.csv"
    with open(p, "w", newline="") as f:
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HEADER)
        for lid, metric, unit, value in [(0, "dram__bytes_read.sum", "Mbyte", "500"),
                                         (0, "gpu__time_duration.sum", "usecond", "100"),
                                         (1, "dram__bytes_write.sum", "byte", "7"),
                                         (1, "gpu__time_duration.sum", "usecond", "300")]:
            w.writerow([lid, 1, "python", "h", "void ctd::k_a(int)", 1, 7, "(256, 1, 1)",
                        "(152, 1, 1)", 0, "10.3", "Command line profiler metrics", metric, unit,
                        value])
    out = measure.ncu_launch_summary(str(p)).splitlines()
    row = out[1].split()
    assert row[0] == "ctd::k_a" and row[1] == "2" and float(row[2]) == pytest.approx(0.4)
