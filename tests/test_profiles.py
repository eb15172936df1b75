"""The committed ncu summaries stay consistent with what the benchmark reports:
the summary the traffic constant points to names the same kernel source hash
and the same byte count, and every summary's command runs committed files
only (no scratch paths)."""
from __future__ import annotations

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_profiles", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_constant_matches_its_summary():
    nt = _bench().NCU_TRAFFIC
    path = os.path.join(ROOT, nt["summary"])
    text = open(path, encoding="utf-8").read()
    assert f"sha256 prefix {nt['sha256_prefix']}" in text
    assert nt["source"] in text
    m = re.search(r"traffic per launch \(read \+ write\) \| ([0-9,]+) B", text)
    assert m, "the summary states the traffic per launch"
    assert int(m.group(1).replace(",", "")) == nt["bytes"]


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md")))
def test_profile_commands_run_committed_files(name):
    text = open(os.path.join(ROOT, "profiles", name), encoding="utf-8").read()
    assert "Command" in text, "each summary gives the command that made it"
    assert "_work/" not in text
    for script in re.findall(r"python3? ([\w./-]+\.py)", text):
        assert os.path.exists(os.path.join(ROOT, script)), script
