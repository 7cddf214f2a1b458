"""The reference arm of bench.py (the FP64 oracle's chain, CPU only) prints the
benchmark's JSON line: the requested steps on a small workload, with the
counts it ran, a cpu_baseline and an e2e entry.  Under torchrun only rank 0
prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, env=env, timeout=600, check=True)
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_line_on_the_tiny_workload():
    lines = _run(None, "--workload", "1", "--steps", "4", "--warmup", "2")
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 4 and d["warmup"] == 2 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["value"] * d["ms_per_step"] - 1e3) < 1e-6 * 1e3
    assert d["unit"] == "steps/s" and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["steps"] == 4
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "tiny-200ev-analytic"


def test_reference_arm_other_ranks_print_nothing():
    lines = _run({"RANK": "1", "WORLD_SIZE": "1"}, "--workload", "1", "--steps", "2", "--warmup", "1")
    assert lines == []
