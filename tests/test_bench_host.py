"""Host-side pieces of bench.py (CPU): workload descriptions, the measured-peak lookup,
the committed ncu traffic figure and the command line."""
import json
import sys

import pytest

import bench


def test_workloads_and_units():
    wl = bench.make_workload("batch256", 0, steps=3)
    assert len(wl.sheets) == 256 and wl.steps == 3
    assert bench.units_per_step(wl) == sum(s.n for s in wl.sheets) * 3
    cfg = bench.workload_config(wl, "batch256")
    assert cfg["sheets"] == 256 and cfg["time_steps"] == 3 and "workload" in cfg
    other = bench.make_workload("batch256", 1, steps=3)  # another rank: another seeded batch
    assert [s.n for s in other.sheets[:16]] != [s.n for s in wl.sheets[:16]]
    assert all(s.forces is None or s.forces.shape[0] == 3 for s in wl.sheets)


def test_measured_peak_reads_the_peaks_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.6}))
    assert bench.measured_peak() == (6789.6, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")


def test_committed_traffic_is_the_summary_line():
    t = bench.committed_traffic()
    assert t is not None and 2.0e8 < t < 2.5e8  # one full-matrix SpMV launch of the batch
    # the roofline kernel of the line: one whole CG solve of the batch (129.6 GB of
    # algorithmic bytes, mostly served from L2)
    w = bench.committed_traffic("cg_solve")
    assert w is not None and 1.0e8 < w < 1.296e11


def test_command_line_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    a = bench.parse()
    assert a.impl == "reference" and a.steps == 2
