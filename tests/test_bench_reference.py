"""CPU check of bench.py's reference arm (--impl reference): the FP64 oracle on the host, one JSON line with
the contract's keys. The sample grid is shrunk to 16 x 17 x 16 so that the check takes seconds."""
import json
import sys

import pytest


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    import bench
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 16)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "16x17x16" in d["cpu_baseline"]["sample"]


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    """Under torchrun every rank but 0 exits without work and prints nothing."""
    import bench
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 16)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                      "--warmup", "1"])
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main()
    assert capsys.readouterr().out.strip() == ""
