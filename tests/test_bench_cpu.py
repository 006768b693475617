"""Host logic of bench.py (no GPU): the algorithmic bytes per stage behind the
roofline line, the DRAM-traffic lookup keyed by the workload and the hash of
the stage's kernel sources, the measured-peak lookup and its fallback, and the
command-line defaults the measurement contract asks for."""
import json
import sys

import pytest

import bench


def test_fft_pass_bytes_are_one_read_and_one_write_of_the_mesh():
    b = bench.stage_bytes(3000, (64, 64, 64), 64, 50, 4, 188746)
    assert b["fft"] == 2 * 64 ** 3 * 64 * 4 == 134217728          # 134 MB per pass at 3000 atoms, mesh 64^3
    assert b["force_fft"] == 2 * b["fft"]                           # the force mesh holds two vectors per probe
    assert b["prologue"] == 3 * 3000 * 64 * (4 * 8 + 4)             # l, y_k-1, y_k-2 in, y* out (FP64), d out (FP32)
    assert bench.stage_bytes(3000, (64, 64, 64), 64, 50, 8, 188746)["fft"] == 2 * b["fft"]


def test_source_hash_is_stable_and_per_stage():
    h = bench.source_hash(bench.STAGE_SOURCES["fft"])
    assert h == bench.source_hash(bench.STAGE_SOURCES["fft"]) and len(h) == 12
    assert bench.source_hash() != h          # all of csrc, not only the FFT stage's files


def test_dram_traffic_lookup(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    cur = bench.source_hash(bench.STAGE_SOURCES["fft"])
    prof = tmp_path / "profiles"
    prof.mkdir()
    f = prof / "dram_traffic.txt"
    f.write_text("# stage workload bytes sources\n"
                 f"fft water 123 {cur}\n"
                 f"fft other 7 {cur}\n")
    assert bench.dram_traffic("fft", "water") == 123.0
    assert bench.dram_traffic("fft", "unknown") is None
    f.write_text("fft water 123 000000000000\n")                   # taken on other sources: not used
    assert bench.dram_traffic("fft", "water") is None
    f.unlink()
    assert bench.dram_traffic("fft", "water") is None


def test_measured_peaks_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")           # the profiling recipe's fallback
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.0}))
    assert bench.measured_peaks() == (6789.0, "measured")


def test_command_line_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert a.gpus == 1 and a.warmup >= 3 and a.impl == "ours" and a.workload == "water100002"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--choices", "64,7,16,32", "--impl", "reference"])
    a = bench.parse_args()
    assert [int(v) for v in a.choices.split(",")] == [64, 7, 16, 32] and a.impl == "reference"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "bogus"])
    with pytest.raises(SystemExit):
        bench.parse_args()


def test_roofline_line_labels_its_basis(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    stages = {"fft": {"achieved_gbs": 4000.0, "us_per_launch": 500.0}}
    r = bench.roofline(stages, "fft", 8000.0, "measured", "w", 20, npts_bytes=2 * 10 ** 9)
    assert r["frac"] == 0.5 and r["traffic"] is None and "frac_dram" not in r
    assert r["basis"].startswith("algorithmic") and r["mesh_exceeds_l2"]
    cur = bench.source_hash(bench.STAGE_SOURCES["fft"])
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(f"fft w 2000000000 {cur}\n")
    r = bench.roofline(stages, "fft", 8000.0, "measured", "w", 20, npts_bytes=10 ** 6)
    assert abs(r["frac_dram"] - 0.5) < 1e-12 and not r["mesh_exceeds_l2"]


def test_covering_members_of_a_batch_replay():
    order, k = bench.covering_members([5.0, 40.0, 1.0, 30.0, 2.0], 70.0)
    assert list(order[:2]) == [1, 3] and k == 2                      # 40 + 30 reach the 70 ms replay
    assert bench.covering_members([5.0, 40.0, 1.0, 30.0, 2.0], 71.0)[1] == 3
    assert bench.covering_members([1.0, 1.0], 100.0)[1] == 2          # never more than the members
