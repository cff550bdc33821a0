"""The roofline's DRAM traffic in bench.py comes from a committed ncu capture
of exactly the timed kernel: same sources (hash), workload, storage and
kernel shape.  Anything else must give null, never another kernel's bytes."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_committed_record_is_used_only_for_its_sources():
    rec = json.load(open(bench.TRAFFIC_FILE))
    b = bench.traffic_per_launch("fp32", "many_disks", (0, 8, 8))
    if rec["fluid_src_sha"] != bench.fluid_src_sha():
        assert b is None  # sources changed since the capture: reported as null
        return
    assert b is not None and b == rec["bytes_per_launch"]["many_disks/fp32/0,8,8"]
    # DRAM reads cannot be below the algorithmic read (8 populations x 4 B per node)
    assert b > 8 * 4 * 1024 * 4096


def test_other_shapes_storage_or_workloads_give_null():
    assert bench.traffic_per_launch("fp32", "many_disks", (0, 4, 4)) is None
    assert bench.traffic_per_launch("fp32", "many_disks", (4, 8, 8)) is None
    assert bench.traffic_per_launch("fp32", "ensemble", (0, 8, 8)) is None


def test_changed_sources_give_null(tmp_path, monkeypatch):
    rec = json.load(open(bench.TRAFFIC_FILE))
    rec["fluid_src_sha"] = "0" * 16
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_per_launch("fp32", "many_disks", (0, 8, 8)) is None
