"""The benchmark's CPU legs (no GPU): the reference arm's JSON line and the oracle sweep."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["value"] > 0 and j["higher_is_better"] is True
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert j["metric"] == bench.METRIC and j["unit"] == bench.UNIT


def test_reference_arm_other_ranks_print_nothing(capsys, monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out.strip() == ""


def test_cpu_sweep_line(capsys):
    bench.main(["--cpu-sweep", "--cpu-sweep-sizes", "64,128"])
    j = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert [r["n"] for r in j["measured"]] == [64, 128]
    assert all(r["seconds"] > 0 for r in j["measured"])
    assert j["paper_single_core"]["seconds"] == 0.022


def test_traffic_entries_are_keyed_by_source():
    """A traffic entry is used only for the kernel source it was measured on."""
    assert bench.ncu_traffic("no_such_kernel_gmm16k") is None
    h = bench.source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_cpu_baseline_reports_its_extrapolation_as_such():
    b = bench.cpu_baseline("roll64k", n_s=128, n_full=65536)
    assert b["kind"] == "oracle" and b["cores"] == 1 and b["value"] > 0
    assert b["extrapolated"]["n"] == 65536 and "not measured" in b["extrapolated"]["how"]
    assert abs(b["extrapolated"]["seconds"] - 65536 ** 3 / (b["value"] * 1e9)) < 1e-6 * b["extrapolated"]["seconds"]


def test_default_workload_is_the_n65536_roll():
    import argparse  # noqa: F401
    assert "roll64k" in bench.WORKLOAD_TEXT
    src = open(bench.__file__).read()
    assert 'ap.add_argument("--workload", default="roll64k"' in src
