"""Host logic of the benchmark, CPU only: the roofline's byte counts, the clock summary that decides
whether a run is kept, and the source hash that ties a committed ncu traffic figure to the kernels."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_unit_bytes_are_the_per_unit_figures():
    """A lepton-step reads x, p, s (36 B), tau (8) and the id (8) and writes x, p, s, tau (44): 96 B; a
    photon-step reads x, k, P, tau and the id (52) and writes x, P, tau (32): 84 B; a stored daughter
    52 B (x, momentum, spin or P, tau, id)."""
    assert bench.unit_bytes(1, 0, 0) == 36 + 8 + 8 + 44
    assert bench.unit_bytes(0, 1, 0) == 36 + 8 + 8 + 32
    assert bench.unit_bytes(0, 0, 1) == 12 + 12 + 12 + 8 + 8
    assert bench.unit_bytes(3, 5, 7) == 3 * 96 + 5 * 84 + 7 * 52


def test_design_bytes_are_below_the_per_unit_figures():
    """The layout's own traffic: 88 B per lepton-step (the id only at events), 56 B per photon-step
    without a pair rate (read 44, write x 12), 76 B with one, 8 B per event, 52 B per stored daughter;
    never above the per-unit figures for a step in which every event stores its daughter."""
    assert bench.design_bytes(1, 0, 0, 0, 0) == 44 + 44
    assert bench.design_bytes(0, 1, 0, 0, 0) == 44 + 12
    assert bench.design_bytes(0, 1, 1, 0, 0) == 44 + 12 + 20
    for lep, pho, rate in ((10, 0, 0), (0, 10, 10), (5, 100, 30)):
        ev = lep // 2
        assert bench.design_bytes(lep, pho, rate, ev, ev) <= bench.unit_bytes(lep, pho, ev)


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary():
    """Median SM clock under load, the maximum, and every throttle reason seen active (a run with a
    hardware or thermal slowdown is rejected by the rules it is measured under; the power cap is noted)."""
    lines = [_line(2070, 2070)] * 5 + [_line(1900, 2070, cap="Active")] + ["garbage", ""]
    s = bench.summarize_clocks(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 6
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.summarize_clocks([_line(1500, 2070, hw="Active"), _line(1500, 2070, hwt="Active")])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and s["sm_mhz"] == 1500.0
    assert bench.summarize_clocks(["nothing here"]) is None


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    """The hash that keys the committed ncu traffic figure covers code lines only: rewording a comment
    keeps it, changing code does not."""
    src = tmp_path / "paper_2511_08929_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (src / f).write_text("int a = 1;  // one\n\n// a note\nint b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    for f in bench.KERNEL_SOURCES:
        (src / f).write_text("int a = 1;  // another wording\n// a longer note\n\nint b = 2;\n")
    assert bench.kernel_source_hash() == h0
    (src / bench.KERNEL_SOURCES[0]).write_text("int a = 3;\nint b = 2;\n")
    assert bench.kernel_source_hash() != h0


def test_traffic_figure_is_keyed_to_its_sources(tmp_path, monkeypatch):
    """bench.py uses the committed traffic figure only while the kernel sources hash as they did when it
    was captured; otherwise the line's traffic is null."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_2511_08929_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (src / f).write_text("int x;\n")
    d = {"dram_bytes_per_particle_step": 76.0, "source_sha256": bench.kernel_source_hash(), "source": "test"}
    (prof / "batch_step_kernel_traffic.json").write_text(json.dumps(d))
    assert bench.measured_traffic()["dram_bytes_per_particle_step"] == pytest.approx(76.0)
    (src / bench.KERNEL_SOURCES[1]).write_text("int y;\n")
    assert bench.measured_traffic() is None
