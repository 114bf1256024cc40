"""Host-side parts of the benchmark (no GPU): the reference arm's JSON line,
the recorded DRAM traffic that must go stale when the measured kernel's
source changes, and the per-kernel algorithmic bytes."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "random-1m", "--steps", "1", "--warmup", "0", "--ref-iters", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["config"]["workload"] == "random-1m"


def test_kernel_text_ends_with_the_kernel():
    path = os.path.join(ROOT, "paper_1705_02313_gb300", "csrc", "pg_iter.cu")
    text = bench.kernel_text(path, "k_chain1(")
    whole = open(path, "rb").read()
    assert whole.startswith(text) and text.rstrip().endswith(b"}")
    assert b"k_chain1(" in text and b"k_scatter(int32_t" not in text  # later kernels are not part of it
    body = text[text.index(b"{", text.index(b"k_chain1(")):]
    assert body.count(b"{") == body.count(b"}")  # the kernel's body is complete


def test_recorded_traffic_goes_stale_with_the_kernel_source(tmp_path, monkeypatch):
    # a copy of the sources and of the recorded traffic: valid as committed, stale after an edit of the
    # kernel, still valid after an edit below it
    for d in ("paper_1705_02313_gb300/csrc", "profiles"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = json.load(open(tmp_path / "profiles" / "traffic.json"))["random-10m"]["classify"]
    rec["source_hash"] = bench.kernel_source_hash("chain1")
    json.dump({"random-10m": {"chain1": rec}}, open(tmp_path / "profiles" / "traffic.json", "w"))
    assert bench.measured_traffic("chain1", "random-10m") == rec["dram_bytes_per_launch"]
    src = tmp_path / "paper_1705_02313_gb300" / "csrc" / "pg_iter.cu"
    text = src.read_text()
    src.write_text(text + "\n// a comment after every kernel\n")
    assert bench.measured_traffic("chain1", "random-10m") == rec["dram_bytes_per_launch"]
    i = text.index("k_chain1(")
    j = text.index("{", i)
    src.write_text(text[:j + 1] + "\n    // an edit inside the kernel\n" + text[j + 1:])
    assert bench.measured_traffic("chain1", "random-10m") is None
    assert bench.measured_traffic("sink_scan", "random-10m") is None  # nothing recorded


def test_algorithmic_bytes_of_the_passes():
    s = {"n": 100, "m": 300, "n_odd": 40, "m_odd": 150, "n_even": 60, "m_even": 150}
    assert bench.algorithmic_bytes("chain1", s) == 15 * 100
    assert bench.algorithmic_bytes("walk", s) == 9 * 100
    assert bench.algorithmic_bytes("classify", s) == 10 * 100
    assert bench.algorithmic_bytes("switch_odd", s) == 12 * 40 + 8 * 150
    assert bench.algorithmic_bytes("sink_scan", s) == 8 * 100
    assert bench.algorithmic_bytes("no_such_kernel", s) is None
