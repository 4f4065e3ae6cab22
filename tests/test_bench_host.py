"""Host arithmetic of bench.py on CPU: the source-hash gate of the committed ncu records (a record
counts only while the kernel sources it names are unchanged), the on-chip roofline's byte count
and peak, and the committed records' own form."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_record_gate(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_bytes(b"kernel one\n")
    (tmp_path / "b.cuh").write_bytes(b"header\n")
    sha = hashlib.sha256(b"kernel one\n" + b"header\n").hexdigest()
    rec = {"sources": ["a.cu", "b.cuh"], "source_sha256": sha, "dram_bytes_read_per_solve": 100,
           "dram_bytes_write_per_solve": 23}
    (tmp_path / "profiles" / "cfr_full_game_seed5.traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("full_game", 5) == 123
    assert bench.recorded_traffic("full_game", 6) is None  # no record
    (tmp_path / "a.cu").write_bytes(b"kernel two\n")  # the kernel changed since the capture
    assert bench.recorded_traffic("full_game", 5) is None
    rec["sources"] = ["b.cuh", "a.cu"]  # the hash runs over the sources in the record's order
    rec["source_sha256"] = hashlib.sha256(b"header\n" + b"kernel two\n").hexdigest()
    (tmp_path / "profiles" / "cfr_full_game_seed5.traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("full_game", 5) == 123


def test_onchip_roofline(monkeypatch):
    monkeypatch.setattr(bench, "_record", lambda name: None)
    assert bench.onchip_roofline(10, 0, 1.0, 2000.0, 152) is None
    assert bench.onchip_roofline(10, 5, 0.0, 2000.0, 152) is None
    r = bench.onchip_roofline(swept=1_000_000, pairs=250_000, kernel_ms=2.0, sm_mhz=2000.0, n_sms=152)
    moved = 28 * 1_000_000 + 32 * 250_000
    assert r["bytes_per_step"] == moved
    assert r["achieved"] == pytest.approx(moved / 2e-3 / 1e9)
    assert r["peak"] == pytest.approx(128 * 152 * 2000e6 / 1e9)  # 38.9 TB/s at 2 GHz
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "smem" and "ncu" not in r


def test_committed_records_are_well_formed():
    d = os.path.join(ROOT, "profiles")
    recs = [f for f in os.listdir(d) if f.endswith(".json")]
    assert recs
    for f in recs:
        rec = json.load(open(os.path.join(d, f)))
        assert rec.get("command", "").startswith(("ncu ", "PASUR_VERBOSE=1 ncu ")), f
        assert "--clock-control none" in rec["command"], f
        if "sources" in rec:
            assert len(rec["source_sha256"]) == 64, f
            for s in rec["sources"]:
                assert os.path.exists(os.path.join(ROOT, s)), (f, s)
