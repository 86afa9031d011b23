"""The checked build (-DTPX_CHECKED, libtpx_checked.so): the fused kernel
tests every data-dependent index (hash chains, member lists, roots, cluster
ids, output positions) against its array and reports a violation in the
status word instead of touching memory -- the stand-in for a sanitizer. On
the parity workloads it reports none, and its results equal the oracle's.
Runs in a subprocess: a process loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r"""
import sys
sys.path[:0] = [ROOT, HERE]
import paper_2603_04942_gb300 as tpx
from paper_2603_04942_gb300 import build
tpx.load(build.build(checked=True))
import synth
from gpu_common import assert_parity, gpu_run, oracle_run
ST_BOUNDS = 1 << 8
small = synth.generate(synth.small(n_shots=300, pair_frac=0.3, dark_per_shot=2.0))[0]
dense = synth.generate(synth.small(n_shots=100, particles_per_shot=200.0, pair_frac=0.5))[0]
high = synth.generate(synth.streaming(10e6, 12))[0]
cases = [
    ("cc 4096 tiles", small, dict(tile=tpx.TILE_4096), {}),
    ("cc 2048 tiles", small, dict(tile=tpx.TILE_2048), {}),
    ("paper mode", small, dict(mode=tpx.MODE_PAPER), dict(mode=tpx.MODE_PAPER)),
    ("radius 3", small, dict(rx=3, ry=3), dict(rx=3, ry=3)),
    ("dense shots", dense, {}, {}),
    ("shots beyond a range (redo)", high, dict(tof_max=synth.STREAM_TOF_MAX_TICKS),
     dict(tof_max=synth.STREAM_TOF_MAX_TICKS)),
]
for name, pk, gkw, okw in cases:
    g = gpu_run(pk, **gkw)
    assert g["status"] == 0, (name, g["status"])
    assert not (g["counters"]["status_bits"] & ST_BOUNDS), name
    assert_parity(g, oracle_run(pk, **okw))
    print("ok", name, flush=True)
"""


def test_checked_build_reports_no_violation_and_matches_the_oracle():
    code = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("ok ") == 6


PHASE_SCRIPT = r"""
import sys
sys.path[:0] = [ROOT, HERE]
import paper_2603_04942_gb300 as tpx
from paper_2603_04942_gb300 import build
tpx.load(build.build(phases=True))
import synth
from gpu_common import assert_parity, gpu_run, oracle_run
# across the first pixel wrap: the wrap step into a range's first pixel
pk = synth.generate(synth.large(n_shots=2000))[0]
for tile in (tpx.TILE_2048, tpx.TILE_4096):
    g = gpu_run(pk, tile=tile)
    assert g["status"] == 0 and g["counters"]["redone"] == 0, (tile, g["status"], g["counters"])
    assert_parity(g, oracle_run(pk))
    print("ok", tile, flush=True)
"""


def test_phase_timing_build_matches_the_oracle_without_a_redo():
    """The instrumented build's timers shift the warps' timing: it once
    exposed a read of a packet another thread had already replaced by its
    record (the wrap step into a range's first pixel). Its results must equal
    the oracle's with no call handed to the general path."""
    code = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + PHASE_SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("ok ") == 2


def test_phase_timing_build_counts_every_phase():
    """The instrumented build (-DTPX_PHASE_TIMING) runs the same kernel with
    per-phase cycle counters; every phase of a tile is counted once."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--phase-shares", "3000", "--tile", "2048"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sh = d["shares"]
    assert abs(sum(sh.values()) - 1.0) < 1e-3
    for k in ("neighbour pass", "walk 4 (records)", "unions", "tile load"):
        assert sh[k] > 0, k


BATCH_SCRIPT = r"""
import sys
sys.path[:0] = [ROOT, HERE]
import paper_2603_04942_gb300 as tpx
from paper_2603_04942_gb300 import build
tpx.load(build.build(checked=True))
from test_gpu_batch import _concat, _ion_runs, check_against_oracle, run_batch
ST_BOUNDS = 1 << 8
pk, offs = _concat(_ion_runs(51, 3, (350, 500), shots=(3, 6)))
for tile in (tpx.TILE_4096, tpx.TILE_2048):
    g = run_batch(pk, offs, tile=tile)
    assert g["counters"]["redone"] == 0, g["counters"]
    assert not (g["counters"]["status_bits"] & ST_BOUNDS), tile
    check_against_oracle(g, pk, offs)
    print("ok", tile, flush=True)
"""


def test_checked_build_big_ranges_in_a_batch():
    """The big-range path of a batch (shots of 12k-18k pixels, both tile
    geometries) under the checked build: no index outside its array, nothing
    redone, results equal to the oracle's run by run."""
    code = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + BATCH_SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("ok ") == 2
