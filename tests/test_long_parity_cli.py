"""CPU: the long-parity runner's oracle-only mode (tests/long_parity.py --no-gpu --sensitivity).

On the 32 x 33 x 32 workload for 3 RK steps it writes its JSON record, and the oracle started from the
state moved by about one rounding unit stays within a few hundred rounding units of the unperturbed run
(the growth the runner reports for the large workloads is a property of those, not of the tool).
"""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_sensitivity_mode_on_the_small_workload(tmp_path):
    out = tmp_path / "p.json"
    r = subprocess.run([sys.executable, os.path.join(HERE, "long_parity.py"), "--workload", "rt32", "--steps", "3",
                        "--check", "1", "3", "--sensitivity", "--no-gpu", "--out", str(out)],
                       capture_output=True, text=True, timeout=600, cwd=os.path.dirname(HERE))
    assert r.returncode == 0, r.stderr[-2000:]
    rec = json.loads(out.read_text())
    assert rec["workload"] == "rt32" and set(rec["steps"]) == {"1", "3"}
    for step in ("1", "3"):
        d = rec["steps"][step]["perturbed_oracle_vs_oracle"]
        assert set(d) == {"z", "om", "m2", "m1", "m3"}
        assert 0 < max(d.values()) < 1e-13
        assert "fp64_vs_oracle" not in rec["steps"][step]
