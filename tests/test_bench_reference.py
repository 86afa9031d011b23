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


def _fake_outputs(pk, o):
    """Device-output stand-ins (CPU tensors) holding the oracle's own result
    of the whole stream, laid out as tpx_process writes them."""
    import numpy as np
    import torch
    import paper_2603_04942_gb300 as tpx
    cl = np.ascontiguousarray(o["clusters"].astype(tpx.CLUSTER_DTYPE))
    return dict(labels=torch.from_numpy(o["labels"].copy()),
                clusters=torch.from_numpy(np.frombuffer(cl.tobytes(), np.uint8).copy()),
                trig=torch.from_numpy(o["triggers"].copy()))


def test_sampled_parity_check_accepts_equal_and_rejects_planted_mismatch():
    """The benchmark's sampled oracle check of the timed call: shot ranges
    cut at TDC packets, regenerated, run through the oracle from their wrap
    counts and compared with the whole call's outputs. Given the oracle's own
    whole-stream result it passes; a record changed in that copy (a mistake
    planted on the CPU) makes it fail."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    p = synth.large(n_shots=2500)
    pk = synth.generate(p)[0]
    o = oracle.run(pk, oracle.Config())
    assert o["status"] == 0
    h_pk = torch.from_numpy(pk.view(np.int64).copy())
    out = _fake_outputs(pk, o)
    n_cl = o["clusters"].size
    r = bench.parity_sampled(p, h_pk, h_pk, out, n_cl, 2500, 800)
    assert r["ok"] is True, r
    assert [x["shots"] for x in r["ranges"]] == [[0, 800], [1700, 2500]]
    assert r["records"] > 1000 and r["labels"] > 10 * r["records"]
    # plant a mistake in one record of the last range
    bad = o["clusters"].copy()
    j = int(np.flatnonzero(bad["shot"] == 2000)[0])
    bad["s_x"][j] += 1
    o2 = dict(o, clusters=bad)
    r2 = bench.parity_sampled(p, h_pk, h_pk, _fake_outputs(pk, o2), n_cl, 2500, 800)
    assert r2["ok"] is False and r2["ranges"][0]["ok"] and not r2["ranges"][1]["ok"]
    # and one label of the first range
    lab = o["labels"].copy()
    q = int(np.flatnonzero(lab >= 0)[100])
    lab[q] += 1
    r3 = bench.parity_sampled(p, h_pk, h_pk, _fake_outputs(pk, dict(o, labels=lab)), n_cl, 2500, 800)
    assert r3["ok"] is False and not r3["ranges"][0]["ok"]
