"""The benchmark's reference arm (the oracle on the host cores) runs on the
CPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--ref-shots", "300", "--shots", "2000"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_cpu_baselines_on_small_samples():
    """Both CPU-baseline legs of the line (single-threaded, and one process
    per core started together) run on small samples of the workload."""
    sys.path.insert(0, ROOT)
    import bench
    sys.argv = ["bench.py", "--shots", "4000"]
    args = bench.parse()
    one = bench.cpu_baseline(args, 300)
    allc = bench.cpu_baseline_parallel(args, 200)
    assert one["cores"] == 1 and one["value"] > 0 and one["kind"] == "oracle"
    assert allc["cores"] >= 1 and allc["value"] > 0 and "processes" in allc["sample"]
