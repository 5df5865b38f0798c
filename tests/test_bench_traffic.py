"""bench.py reports the dominant kernel's ncu DRAM traffic only from a capture
of that same kernel: the stored record must match the node label, the storage
type and the hash of the kernel's sources, else the traffic is null."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("sift3d_bench_traffic", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_record_is_keyed(tmp_path, monkeypatch):
    b = _bench()
    with open(b.TRAFFIC_FILE) as f:
        rec = json.load(f)
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert rec["storage"] in ("f32", "f16", "bf16")
    rec["source_hash"] = b.kernel_source_hash()      # as if just captured
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(p))
    assert b.measured_traffic(rec["label"], rec["storage"]) == float(rec["dram_bytes_per_launch"])
    other = "f16" if rec["storage"] != "f16" else "f32"
    assert b.measured_traffic(rec["label"], other) is None
    assert b.measured_traffic("o1.d3.peak", rec["storage"]) is None


def test_traffic_record_goes_stale_with_the_sources(tmp_path, monkeypatch):
    b = _bench()
    with open(b.TRAFFIC_FILE) as f:
        rec = json.load(f)
    rec["source_hash"] = "0" * 16
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(p))
    assert b.measured_traffic(rec["label"], rec["storage"]) is None
