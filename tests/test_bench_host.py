"""Host-side checks of the benchmark's measurement helpers (no GPU): the clock
summary keeps only samples taken inside the timed region and reports throttle
reasons, and the profile check hashes code, not comments."""
import os
import stat
import time

import bench

FAKE = """#!/bin/bash
# stand-in for the sampler: {n_before} rows at {low} MHz, then rows at {high} MHz
i=0
while true; do
  if [ $i -lt {n_before} ]; then c={low}; else c={high}; fi
  echo "0, $c, 2070, 200.0, 0x0, {hw}, Not Active, Not Active, Not Active"
  i=$((i+1)); sleep 0.02
done
"""


def _fake_smi(tmp_path, monkeypatch, n_before=10, low=900, high=2070, hw="Not Active"):
    d = tmp_path / "bin"
    d.mkdir()
    p = d / "nvidia-smi"
    p.write_text(FAKE.format(n_before=n_before, low=low, high=high, hw=hw))
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(d) + os.pathsep + os.environ["PATH"])


def test_clock_summary_keeps_the_timed_region(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.Clocks(0)
    c.start()
    deadline = time.monotonic() + 5
    while len(c.lines) < 12 and time.monotonic() < deadline:  # past the low-clock rows
        time.sleep(0.01)
    c.mark_begin()
    time.sleep(0.2)
    c.mark_end()
    out = c.stop()
    assert out["window"] == "timed region"
    assert out["samples"] >= 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_clock_summary_reports_throttle_reasons(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch, n_before=0, hw="Active")
    c = bench.Clocks(0)
    c.start()
    c.mark_begin()
    time.sleep(0.1)
    c.mark_end()
    out = c.stop()
    assert out["reasons"] == ["hw_slowdown"]


def test_clock_summary_without_a_sampler(monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    c = bench.Clocks(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_kernel_hash_ignores_comments_and_blank_space(tmp_path, monkeypatch):
    src = tmp_path / "paper_1603_08390_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (src / name).write_text("int f(int x) {\n  return x + 1;  // one\n}\n/* block */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_sha()
    for name in bench.KERNEL_SOURCES:
        (src / name).write_text("int f(int x)   { return x + 1; }  // another comment\n")
    assert bench.kernel_source_sha() == h1
    (src / bench.KERNEL_SOURCES[0]).write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_sha() != h1
