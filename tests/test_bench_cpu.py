"""The bench's command-line contract on CPU: its defaults (one GPU, at least three warm-up
steps) and the reference arm (the oracle on the host cores), which must print one JSON line
with the keys of the benchmark line (impl, value, unit, steps, cpu_baseline, e2e, config)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_defaults():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        args = bench.parse()
    finally:
        sys.argv = old
    assert args.gpus == 1 and args.impl == "ours" and args.warmup >= 3 and args.steps >= 1
    assert args.workload == 4 and args.case == "full"


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--case", "small", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mrays/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_reference_arm_config_equals_ours():
    """Both arms print the same `config` object, so their lines describe one workload."""
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    sys.argv = ["bench.py", "--case", "small"]
    try:
        args = bench.parse()
    finally:
        sys.argv = old
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--case", "small", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][0])
    assert d["config"] == bench.bench_config(bench.make_workload(args), 1)
