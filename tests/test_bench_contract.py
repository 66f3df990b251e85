"""The benchmark's reference arm (the FP64 oracle on the host cores) and its
JSON line, run on the CPU: one line with the metric, unit and direction of
the GPU arm, the cpu_baseline and e2e objects, and nothing from ranks other
than 0.  The GPU arm's line is checked on the GPU by running bench.py."""
from __future__ import annotations

import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def run_reference(env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    if env_extra:
        env.update(env_extra)
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--cpu-chains", "1"], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    return out


def test_reference_arm_prints_one_contract_line():
    out = run_reference()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == bench.UNIT
    assert cb["cores"] >= 1 and "sample" in cb
    e2e = d["e2e"]
    assert e2e == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    out = run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_defaults_meet_the_timing_rules():
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = argv
    assert a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1


@pytest.mark.parametrize("threads", [1, 2])
def test_oracle_sample_rate_is_positive(threads):
    rate, dt = bench.oracle_sample(4, 1, threads)
    assert rate > 0 and dt > 0
