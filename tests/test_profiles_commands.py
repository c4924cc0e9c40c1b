"""Every bench.py command quoted in the ncu summaries under profiles/ parses with bench.py's own argument
parser and names a workload of the input module: the summaries give commands that run committed files."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^&|>\"\n]*)", text):
            out.append((os.path.basename(path), m.group(1).strip()))
    return out


def test_every_summary_names_its_command():
    names = {os.path.basename(p) for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))}
    with_cmd = {n for n, _ in _commands()}
    assert names and names == with_cmd, names - with_cmd


@pytest.mark.parametrize("name,args", _commands())
def test_quoted_bench_command_parses(name, args, monkeypatch):
    import bench
    from paper_2206_09878_gb300.rt_inputs import WORKLOADS
    words = [w for w in shlex.split(args) if not w.startswith("$")]
    monkeypatch.setattr(sys, "argv", ["bench.py", *words])
    a = bench.parse()
    assert a.workload in WORKLOADS, (name, a.workload)
