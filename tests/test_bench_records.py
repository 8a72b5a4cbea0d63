"""The bench's use of committed ncu records: a record counts only while the
hash of the kernel sources it names matches the files (stale -> null), and
the ALU object is FLOP per node x node rate against SMs x 128 lanes x 2 x clock."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, src_text):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "k.cu").write_text(src_text)
    digest = hashlib.sha256(src_text.encode()).hexdigest()
    recs = [{"kernel": "kern", "precision": "fp32", "sources": ["k.cu"], "sources_sha256": digest,
             "bytes_per_launch_full": 123.0, "fp32_flop_per_node": 400.0}]
    (root / "profiles" / "traffic.json").write_text(json.dumps(recs))
    (root / "profiles" / "fp32_ops.json").write_text(json.dumps(recs))
    return root


def test_record_valid_then_stale(tmp_path, monkeypatch):
    root = _tree(tmp_path, "kernel source v1")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_record("kern", "fp32") == 123.0
    assert bench.traffic_record("kern", "bf16") is None
    assert bench.traffic_record("other", "fp32") is None
    a = bench.alu_entry("kern", nodes=1000, launch_s=1e-6, sms=148, sm_mhz=2032.0)
    assert abs(a["peak"] - 148 * 128 * 2 * 2032e6 / 1e12) < 1e-9
    assert abs(a["achieved"] - 400.0 * 1000 / 1e-6 / 1e12) < 1e-9
    assert abs(a["frac"] - a["achieved"] / a["peak"]) < 1e-12
    (root / "k.cu").write_text("kernel source v2")  # the kernel changed after the capture
    assert bench.traffic_record("kern", "fp32") is None
    assert bench.alu_entry("kern", 1000, 1e-6, 148, 2032.0) is None


def test_committed_records_name_existing_sources():
    for name in ("traffic.json", "fp32_ops.json"):
        with open(os.path.join(bench.ROOT, "profiles", name)) as f:
            for r in json.load(f):
                for src in r["sources"]:
                    assert os.path.exists(os.path.join(bench.ROOT, src)), src
                assert "--clock-control none" in r["capture"]
