"""The bench's reference arm (one full hot-path step of the FP64 oracle, measured in timed slices on the
host cores): one JSON line with the contract's keys on rank 0, and nothing (exit status 0) on the other
ranks of a multi-process launch.  Run on the small 4x4x4x8 workload, where the oracle's step takes
about a second."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_the_contract_line():
    p = _run({}, "--steps", "4", "--warmup", "1", "--workload", "t_4x4x4x8")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype",
              "data", "config"):
        assert k in d, k
    assert d["config"]["workload"] == "t_4x4x4x8" and d["value"] > 0
    # one measured hot-path step cut into the timed slices: value is their sum, ms_per_step their mean
    t = d["timed"]
    assert t["hot_path_steps"] == 1 and t["slices"] == 4 and len(t["slice_ms"]) == 4
    assert abs(sum(t["slice_ms"]) - d["value"]) <= 1e-9 * d["value"]
    assert abs(d["ms_per_step"] * 4 - d["value"]) <= 1e-9 * d["value"]
    assert "iterations" in d["cpu_baseline"]["sample"] and "scaled" not in d["cpu_baseline"]["sample"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    p = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0",
             "--workload", "t_4x4x4x8")
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
