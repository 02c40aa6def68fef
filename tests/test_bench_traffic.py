"""bench.py reports roofline.traffic from committed ncu summaries only while
they were taken on the current row-kernel sources: these tests check the
lookup on a temporary profiles folder (the hash match, the named workload,
and a workload family scaled by its rows)."""
import json
import os

import bench


def write(root, name, d):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", name), "w") as f:
        json.dump(d, f)


def test_lookup(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    root = str(tmp_path)
    write(root, "a.json", {"workload": "w-100", "dram_bytes_per_launch": 1234, "kernel_sources_sha256_16": h})
    write(root, "b.json", {"family": "fam-", "capture_rows": 1000, "dram_bytes_read_capture": 900,
                           "dram_bytes_write_capture": 100, "kernel_sources_sha256_16": h})
    write(root, "c.json", {"workload": "stale", "dram_bytes_per_launch": 1, "kernel_sources_sha256_16": "0" * 16})
    monkeypatch.setattr(bench, "ROOT", root)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda read=None: h)
    assert bench.profile_traffic("w-100", 100) == 1234.0
    assert bench.profile_traffic("fam-5000", 5000) == 5000.0      # (900 + 100) bytes per 1000 rows
    assert bench.profile_traffic("stale", 1) is None             # taken on other sources
    assert bench.profile_traffic("other", 1) is None


def test_hash_ignores_comments():
    src = {"x": "int a; // one\n/* two */ int b;"}
    names = bench.ROW_KERNEL_SOURCES
    base = bench.kernel_source_hash(read=lambda n: "int a; int b;" if n == names[0] else "")
    same = bench.kernel_source_hash(read=lambda n: src["x"] if n == names[0] else "")
    other = bench.kernel_source_hash(read=lambda n: "int a; int c;" if n == names[0] else "")
    assert base == same != other
