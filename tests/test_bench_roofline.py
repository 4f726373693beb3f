"""bench.py's roofline block (CPU): the DRAM traffic and the on-chip ceilings
of the committed ncu summary are reported only while the summary was taken on
the kernel source being run (its sha256) and only for the full-size node it
describes; otherwise they are null, so counters of another kernel or another
node size are never reported as this run's."""
import hashlib
import json

import pytest


@pytest.fixture()
def bench(monkeypatch, tmp_path):
    import bench as B
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel source\n")
    rec = {"source": "kernel.cu", "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
           "dram_bytes_per_launch": 1000, "shared_wavefronts_per_launch": 148 * 2032 * 1000,
           "warp_instructions_per_launch": 4 * 148 * 2032 * 1000, "sms": 148, "summary": "profiles/x.md"}
    (tmp_path / "profiles" / "k_hist_staged_root_4m.json").write_text(json.dumps(rec))
    monkeypatch.setattr(B, "ROOT", str(tmp_path))
    return B, src


def test_summary_used_when_the_source_matches(bench):
    B, _ = bench
    r = B.roofline_block(500.0, 6500.0, "measured", 1000, 2.0, {"sm_mhz": 2032.0})
    assert r["traffic"] == 1000
    # 148 * 2032e3 wavefronts per ms at one per SM per clock: 1 ms of the 2 ms launch
    assert r["ceilings"]["shared_pipe"]["floor_ms"] == pytest.approx(1.0)
    assert r["ceilings"]["shared_pipe"]["frac"] == pytest.approx(0.5)
    assert r["ceilings"]["issue"]["floor_ms"] == pytest.approx(1.0)
    assert r["frac"] == pytest.approx(500.0 / 6500.0)


def test_summary_dropped_when_the_source_changed(bench):
    B, src = bench
    src.write_text("// the kernel changed\n")
    r = B.roofline_block(500.0, 6500.0, "measured", 1000, 2.0, {"sm_mhz": 2032.0})
    assert r["traffic"] is None and "ceilings" not in r and "traffic_note" in r


def test_summary_dropped_for_another_node_size(bench):
    B, _ = bench
    r = B.roofline_block(500.0, 6500.0, "measured", 1000, 2.0, {"sm_mhz": 2032.0}, full_size=False)
    assert r["traffic"] is None and "ceilings" not in r and "full-size" in r["traffic_note"]

