"""Host logic of bench.py's DRAM-traffic table (no GPU): an ncu CSV of one captured launch
becomes bytes per launch = dram__bytes_read.sum + dram__bytes_write.sum, stamped with the
hash of the kernel's sources, and bench.py reports that figure only while the sources are
unchanged."""
import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEADER = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
          "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _write_capture(path, read, write, ns):
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(HEADER)
        for name, unit, value in (("dram__bytes_read.sum", "byte", f"{read:,}"),
                                  ("dram__bytes_write.sum", "byte", f"{write:,}"),
                                  ("gpu__time_duration.sum", "ns", str(ns))):
            w.writerow(["0", "1", "python3", "127.0.0.1", "kernel(args)", "1", "13", "(608, 1, 1)", "(256, 1, 1)",
                        "0", "10.3", "Command line profiler metrics", name, unit, value])


def test_record_traffic_sums_read_and_write(tmp_path):
    _write_capture(tmp_path / "dram_3d_x6_cs.csv", 717_800_000, 599_500_000, 241056)
    out = tmp_path / "traffic.json"
    assert bench.record_traffic(str(tmp_path), str(out)) == 0
    tab = json.load(open(out))
    assert list(tab) == ["mrt3d_256:collide_stream@bf16x6split"]  # only the capture present
    rec = tab["mrt3d_256:collide_stream@bf16x6split"]
    assert rec["bytes_per_launch"] == 717_800_000 + 599_500_000
    assert rec["duration_ns"] == 241056
    assert rec["precision"] == "bf16x6split"
    assert rec["source_sha"] == bench.source_sha(rec["sources"])
    assert "paper_1706_09161_gb300/csrc/collide_stream.cu" in rec["sources"]


def test_committed_table_matches_current_sources():
    """Every entry of profiles/traffic.json names existing sources; an entry whose hash no
    longer matches them is reported as unknown (None), never as a stale number."""
    tab = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert set(tab) == set(bench.TRAFFIC_CAPTURES)
    for key, rec in tab.items():
        for src in rec["sources"]:
            assert os.path.exists(os.path.join(ROOT, src)), src
        workload, kernel = key.split("@")[0].split(":")
        got = bench.traffic_for(workload, kernel, rec["precision"])
        fresh = rec["source_sha"] == bench.source_sha(rec["sources"])
        assert got == (rec["bytes_per_launch"] if fresh else None)
