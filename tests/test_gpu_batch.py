"""Batched runs in one launch (tpx_process_batch) against the oracle run on
each run alone: every run is a stream of its own; records and triggers come
run after run with per-run offsets; in CC mode a shot longer than a tile's
range stays in the launch (the big-range path), and runs even that cannot
hold (a range past 65,535 positions; PAPER mode) are redone exactly; empty
runs, one-packet runs, runs starting at odd packets and runs crossing the
pixel wrap are covered."""
import numpy as np
import pytest

import oracle
import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_clusters_equal, oracle_run, to_device
from streams import StreamBuilder

pytestmark = pytest.mark.gpu


def _long_shot_run(rng, pixels=9000, spread=50_000):
    """Three shots; the middle one holds `pixels` pixels at random places,
    their ToF spread over `spread` ticks (the first shot's tile range holds
    two shots)."""
    b = StreamBuilder()
    t = 50_000_000
    for s in range(3):
        b.tdc(t + s * 640_000)
        for _ in range(pixels if s == 1 else 300):
            b.pix(rng.integers(0, 256), rng.integers(0, 256), rng.integers(1, 400),
                  t + s * 640_000 + 800 + rng.integers(0, spread))
    return b.packets()


BEYOND_BIG = 66_000   # pixels of a shot past the big-range path's 65,535 positions


def make_batch(n_runs=20, seed=5, long_shot=True, long_pixels=9000):
    runs = [synth.generate(p)[0] for p in synth.batched(n_runs=n_runs, seed=seed, shots_hi=150, particles_hi=40)]
    rng = np.random.default_rng(seed)
    runs.insert(3, np.zeros(0, np.uint64))                 # an empty run
    runs.insert(5, runs[4][:1].copy())                     # a one-packet run (odd offsets after it)
    runs.insert(8, runs[7][: 2 * 4096 + 3].copy())         # a run cut mid-shot
    if long_shot:
        runs.insert(11, _long_shot_run(rng, long_pixels))  # a shot past a tile's range
    offs = np.zeros(len(runs) + 1, np.int64)
    offs[1:] = np.cumsum([r.size for r in runs])
    pk = np.concatenate(runs) if offs[-1] else np.zeros(0, np.uint64)
    return pk, offs


def run_batch(pk, offs, mode=0, tile=0, labels=True):
    ctx = tpx.Context(tpx.Config(mode=mode, tile_geometry=tile), max_packets=max(1, pk.size))
    try:
        out = ctx.alloc_batch_outputs(pk.size, offs.size - 1, labels=labels, is_peak=labels,
                                      cluster_capacity=max(16, pk.size), trig_capacity=max(16, pk.size))
        ctx.tpx_process_batch(to_device(pk), offs, out)
        rc, cnt = ctx.tpx_sync(check=False)
        return ctx.collect_batch(out, rc, cnt)
    finally:
        ctx.close()


def check_against_oracle(g, pk, offs, mode=0):
    assert g["status"] == 0
    assert g["run_clusters"][-1] == g["n_clusters"] and g["run_trig"][-1] == g["n_trig"]
    labels = []
    for r in range(offs.size - 1):
        a, b = int(offs[r]), int(offs[r + 1])
        o = oracle_run(pk[a:b], mode=mode, index_base=a)
        gc = g["clusters"][g["run_clusters"][r]: g["run_clusters"][r + 1]]
        assert_clusters_equal(gc, o["clusters"])
        assert np.array_equal(g["triggers"][g["run_trig"][r]: g["run_trig"][r + 1]], o["triggers"]), r
        labels.append(o["labels"])
        if g["is_peak"] is not None:
            assert np.array_equal(g["is_peak"][a:b], o["is_peak"]), r
    if g["labels"] is not None:
        assert np.array_equal(g["labels"], np.concatenate(labels))


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_each_run_alone(mode):
    pk, offs = make_batch()
    g = run_batch(pk, offs, mode=mode)
    # the long-shot run: the big-range path in CC mode, the general path in PAPER mode
    assert g["counters"]["redone"] == (0 if mode == 0 else 1)
    check_against_oracle(g, pk, offs, mode)


def test_several_redone_runs_share_one_clustering_pass():
    """Three runs with shots past even the big-range path (more than 65,535
    positions), between ordinary runs: they are redone together (shots kept
    apart per run) and spliced back in run order, with per-packet labels."""
    rng = np.random.default_rng(21)
    pk, offs = make_batch(n_runs=12, seed=8, long_shot=False)
    runs = [pk[offs[r]:offs[r + 1]] for r in range(offs.size - 1)]
    for k, at in enumerate((2, 6, 9)):
        runs.insert(at, _long_shot_run(rng, pixels=BEYOND_BIG + 700 * k))
    offs = np.zeros(len(runs) + 1, np.int64)
    offs[1:] = np.cumsum([r.size for r in runs])
    pk = np.concatenate(runs)
    g = run_batch(pk, offs)
    assert g["counters"]["redone"] == 3
    check_against_oracle(g, pk, offs)


def test_batch_on_the_smaller_tiles():
    pk, offs = make_batch(seed=6)
    g = run_batch(pk, offs, tile=tpx.TILE_2048)
    check_against_oracle(g, pk, offs)


def test_batch_without_redo_and_without_labels():
    pk, offs = make_batch(seed=7, long_shot=False)
    g = run_batch(pk, offs, labels=False)
    assert g["counters"]["redone"] == 0
    check_against_oracle(g, pk, offs)


def test_single_run_batch_equals_tpx_process():
    pk = synth.generate(synth.small(n_shots=300))[0]
    offs = np.array([0, pk.size], np.int64)
    g = run_batch(pk, offs)
    o = oracle.run(pk)
    assert_clusters_equal(g["clusters"], o["clusters"])
    assert np.array_equal(g["labels"], o["labels"])


def test_all_runs_empty():
    pk = np.zeros(0, np.uint64)
    offs = np.zeros(4, np.int64)
    g = run_batch(pk, offs)
    assert g["status"] == 0 and g["n_clusters"] == 0 and g["n_trig"] == 0
    assert np.array_equal(g["run_clusters"], np.zeros(4)) and np.array_equal(g["run_trig"], np.zeros(4))


def test_bad_offsets_rejected():
    import torch
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        out = ctx.alloc_batch_outputs(16, 2)
        d = torch.zeros(16, dtype=torch.int64, device="cuda")
        for offs in (np.array([1, 5, 16]), np.array([0, 9, 5])):
            with pytest.raises(tpx.TpxError):
                ctx.tpx_process_batch(d, offs, out)
    finally:
        ctx.close()


def test_batch_captured_in_a_cuda_graph_replays_exactly():
    """The batched launch captured into a CUDA graph: every replay (run
    tables uploaded, one persistent kernel; the long-shot run redone at
    tpx_sync) gives the eager call's outputs, and eager calls still work
    after the capture."""
    import torch
    pk, offs = make_batch(n_runs=24, seed=9, long_pixels=BEYOND_BIG)
    s = torch.cuda.Stream()
    ctx = tpx.Context(tpx.Config(tile_geometry=tpx.TILE_4096), max_packets=pk.size, stream=s)
    try:
        d = to_device(pk)
        kw = dict(labels=True, is_peak=True, cluster_capacity=max(16, pk.size), trig_capacity=max(16, pk.size))
        with torch.cuda.stream(s):
            ref_out = ctx.alloc_batch_outputs(pk.size, offs.size - 1, **kw)
            out = ctx.alloc_batch_outputs(pk.size, offs.size - 1, **kw)
        ctx.tpx_process_batch(d, offs, ref_out)
        rc, cnt = ctx.tpx_sync(check=False)
        ref = ctx.collect_batch(ref_out, rc, cnt)
        assert rc == 0 and cnt["redone"] >= 1
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            ctx.tpx_process_batch(d, offs, out)
        for _ in range(3):
            with torch.cuda.stream(s):             # the context's stream: tpx_sync waits on it
                out["labels"].fill_(-7)
                g.replay()
            rc, cnt = ctx.tpx_sync(check=False)
            r = ctx.collect_batch(out, rc, cnt)
            assert rc == 0 and cnt["redone"] == ref["counters"]["redone"]
            assert np.array_equal(r["labels"], ref["labels"]) and np.array_equal(r["is_peak"], ref["is_peak"])
            assert np.array_equal(r["run_clusters"], ref["run_clusters"])
            assert np.array_equal(r["run_trig"], ref["run_trig"]) and np.array_equal(r["triggers"], ref["triggers"])
            assert_clusters_equal(r["clusters"], ref["clusters"])
        ctx.tpx_process_batch(d, offs, ref_out)            # an ordinary call after the capture
        rc, cnt = ctx.tpx_sync(check=False)
        assert rc == 0 and np.array_equal(ctx.collect_batch(ref_out, rc, cnt)["labels"], ref["labels"])
    finally:
        ctx.close()


def _ion_runs(seed, n_runs, particles, shots=(4, 12)):
    """Ion-like runs (sigma 1.2 px, ToF 1-20 us, ~36 px per particle) whose
    shots hold `particles` Poisson particles: 10k-20k pixels per shot for
    300-550 particles."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n_runs):
        pp = float(particles[r % len(particles)])
        p = synth.Params(n_shots=int(rng.integers(*shots)), seed=seed * 1000 + r, poisson=True,
                         particles_per_shot=pp, t_start_ticks=int(rng.integers(0, synth.PIX_PERIOD_TICKS)),
                         **synth.ION)
        runs.append(synth.generate(p)[0])
    return runs


def _concat(runs):
    offs = np.zeros(len(runs) + 1, np.int64)
    offs[1:] = np.cumsum([r.size for r in runs])
    return (np.concatenate(runs) if offs[-1] else np.zeros(0, np.uint64)), offs


def _check_counters(g, pk, offs, **okw):
    tot = dict.fromkeys(("kept", "dropped_pre_trigger", "dropped_background", "clusters", "peaks"), 0)
    for r in range(offs.size - 1):
        o = oracle_run(pk[offs[r]:offs[r + 1]], **okw)
        for k in tot:
            tot[k] += int(o["counters"][k])
    for k, v in tot.items():
        assert g["counters"][k] == v, (k, g["counters"][k], v)


@pytest.mark.parametrize("tile", [tpx.TILE_4096, tpx.TILE_2048])
def test_big_shots_stay_in_the_launch(tile):
    """Runs whose shots hold 10k-20k pixels (ion-like, 300-550 particles per
    shot) between ordinary runs: every range past a tile's capacity takes the
    big-range path in the same launch, nothing is redone, and records, labels,
    local maxima, triggers and counters equal the oracle's run by run."""
    runs = _ion_runs(31, 6, (300, 420, 550))
    small = [synth.generate(p)[0] for p in synth.batched(n_runs=6, seed=12, shots_hi=80, particles_hi=40)]
    mixed = [x for pair in zip(runs, small) for x in pair]
    pk, offs = _concat(mixed)
    g = run_batch(pk, offs, tile=tile)
    assert g["counters"]["redone"] == 0
    check_against_oracle(g, pk, offs)
    _check_counters(g, pk, offs)


def test_big_shots_with_a_wider_box_and_radius():
    """The big-range path under rx = ry = 2 and a 64-tick time radius."""
    runs = _ion_runs(33, 3, (350, 500), shots=(3, 6))
    pk, offs = _concat(runs)
    ctx = tpx.Context(tpx.Config(rx=2, ry=2, dt_ticks=64), max_packets=pk.size)
    try:
        out = ctx.alloc_batch_outputs(pk.size, offs.size - 1, labels=True, is_peak=True,
                                      cluster_capacity=pk.size, trig_capacity=pk.size)
        ctx.tpx_process_batch(to_device(pk), offs, out)
        rc, cnt = ctx.tpx_sync(check=False)
        g = ctx.collect_batch(out, rc, cnt)
    finally:
        ctx.close()
    assert g["counters"]["redone"] == 0
    for r in range(offs.size - 1):
        a, b = int(offs[r]), int(offs[r + 1])
        o = oracle_run(pk[a:b], rx=2, ry=2, dt=64, index_base=a)
        assert_clusters_equal(g["clusters"][g["run_clusters"][r]: g["run_clusters"][r + 1]], o["clusters"])
        assert np.array_equal(g["labels"][a:b], o["labels"]) and np.array_equal(g["is_peak"][a:b], o["is_peak"])


def test_big_shot_with_dense_time_bins_and_a_run_past_the_limit():
    """A 12k-pixel shot within 300 ticks (a few wide-open bins: long
    windows), a big shot beside a small one in one tile's range, and a shot
    past the big-range path's limit (that run alone is redone)."""
    rng = np.random.default_rng(41)
    runs = [_long_shot_run(rng, 12_000, spread=300), _long_shot_run(rng, 15_000),
            _long_shot_run(rng, BEYOND_BIG), _ion_runs(35, 1, (450,), shots=(5, 6))[0]]
    pk, offs = _concat(runs)
    g = run_batch(pk, offs)
    assert g["counters"]["redone"] == 1
    check_against_oracle(g, pk, offs)
