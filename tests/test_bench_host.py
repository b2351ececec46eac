"""Host-side pieces of bench.py that need no GPU: algorithmic bytes and the
DRAM-traffic record read back into the roofline."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

NCU_CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","7","python","h","void msrep::csc_direct<msrep::PolF64, 16>(msrep::CscArgs<T1>, const int *, long)","1","7","(256, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","221.84"
"0","7","python","h","void msrep::csc_direct<msrep::PolF64, 16>(msrep::CscArgs<T1>, const int *, long)","1","7","(256, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Kbyte","4,272.13"
"0","7","python","h","void msrep::csc_direct<msrep::PolF64, 16>(msrep::CscArgs<T1>, const int *, long)","1","7","(256, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","297.73"
'''


def test_algorithmic_bytes():
    # CSR: 12 B per FP64 nonzero, 4 B per row pointer, x and y once
    assert bench.algorithmic_bytes("csr", 10, 20, 100, 8, 8) == 1200 + 44 + 160 + 80
    assert bench.algorithmic_bytes("csc", 10, 20, 100, 8, 8) == 1200 + 84 + 160 + 80
    assert bench.algorithmic_bytes("coo", 10, 20, 100, 4, 4) == 1200 + 80 + 40


def test_traffic_record_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "traffic.json"))
    monkeypatch.setattr(bench, "source_stamp", lambda: "stamp-a")
    csv_path = tmp_path / "ncu.csv"
    csv_path.write_text(NCU_CSV)
    e = bench.record_traffic(str(csv_path), "rmat/csc", "ncu ...")
    assert e["kernel"].endswith("csc_direct<msrep::PolF64, 16>")
    assert e["dram_read_bytes"] == 221.84e6
    assert abs(e["dram_write_bytes"] - 4272.13e3) < 1e-6
    assert abs(e["duration_us_under_ncu"] - 297.73) < 1e-9
    assert bench.recorded_traffic("rmat/csc") == e["dram_read_bytes"] + e["dram_write_bytes"]
    assert bench.recorded_traffic("rmat/csr") is None
    # a record taken on other kernel sources does not count
    monkeypatch.setattr(bench, "source_stamp", lambda: "stamp-b")
    assert bench.recorded_traffic("rmat/csc") is None
    assert json.loads((tmp_path / "traffic.json").read_text())["kernels"]["rmat/csc"]["command"] == "ncu ..."


def test_partition_overhead_share():
    # partition 1 ms, SpMV 3 ms -> 25 %; with local pointers 3 ms -> 50 %
    kern = {"rmat/coo": {"call_us": 3000.0}}
    out = bench.partition_overhead({"rmat/coo": 1.0}, {"rmat/coo": 3.0}, kern)["rmat/coo"]
    assert abs(out["pct"] - 25.0) < 1e-12
    assert abs(out["pct_with_local"] - 50.0) < 1e-12
    assert out["spmv_ms"] == 3.0


def test_stamp_ignores_comments_only():
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* no overflow check */\n}\n"
    b = "/* a comment block\n   over lines */\nint f(int x) {\n  return 2 * x;\n}\n"
    c = "int f(int x) {\n  return 3 * x;\n}\n"
    assert bench.code_of(a) == bench.code_of(b)
    assert bench.code_of(a) != bench.code_of(c)
