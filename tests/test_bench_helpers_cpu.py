"""Host helpers of bench.py (no GPU): the peak file and its fallback, and the DRAM traffic
records, which count only while the sources their kernel is built from are unchanged."""
import hashlib
import json

import bench


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0}))
    monkeypatch.setattr(bench, "PEAKS_PATH", str(f))
    p = bench.peaks()
    assert p["_source"] == "measured" and p["hbm_gbs"] == 6000.0
    monkeypatch.setattr(bench, "PEAKS_PATH", str(tmp_path / "missing.json"))
    p = bench.peaks()
    assert p["_source"] == "fallback" and p["hbm_gbs"] == bench.FALLBACK_PEAKS["hbm_gbs"]


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    (tmp_path / "k.cu").write_text("kernel source v1")
    (tmp_path / "k.cuh").write_text("header")
    h = hashlib.sha256()
    for rel in ("k.cu", "k.cuh"):
        h.update((tmp_path / rel).read_bytes())
    rec = {"kern": {"bytes_per_launch": 1234, "sources": ["k.cu", "k.cuh"], "sources_sha": h.hexdigest()[:16]}}
    (tmp_path / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    assert bench.recorded_traffic("kern") == 1234
    assert bench.recorded_traffic("other") is None               # no record for this kernel
    (tmp_path / "k.cu").write_text("kernel source v2")           # the kernel changed since the capture
    assert bench.recorded_traffic("kern") is None
    (tmp_path / "k.cu").unlink()
    assert bench.recorded_traffic("kern") is None


def test_committed_traffic_records_name_existing_sources():
    recs = json.load(open(bench.TRAFFIC_PATH))
    assert recs
    for name, r in recs.items():
        assert r["bytes_per_launch"] > 0, name
        for rel in r["sources"]:
            assert (bench.os.path.exists(bench.os.path.join(bench.ROOT, rel))), (name, rel)
