"""A stream fed as consecutive calls (cut at trigger packets) gives exactly the
single-call result: the unwrap state and trigger count carry over on the
device (chain mode) or through tpx_get_state / tpx_set_state."""
import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_clusters_equal, gpu_run, oracle_run, to_device

pytestmark = pytest.mark.gpu


def run_calls(pk, cuts, chain=True, fused=True):
    import torch
    ctx = tpx.Context(tpx.Config(chain=chain), max_packets=pk.size)
    labels, clusters, trig = [], [], []
    try:
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = pk[a:b]
            d = to_device(part)
            out = ctx.alloc_outputs(part.size, True, True, max(16, part.size), max(16, part.size))
            ctx.tpx_process(d, out, index_base=a)
            rc, cnt = ctx.tpx_sync(check=False)
            assert rc == 0
            r = ctx.collect(out, rc, cnt)
            labels.append(r["labels"])
            clusters.append(r["clusters"])
            trig.append(r["triggers"])
        return np.concatenate(labels), np.concatenate(clusters), np.concatenate(trig), ctx.tpx_get_state()
    finally:
        ctx.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_chained_calls_equal_one_call(seed):
    # shots 480..560 of the small configuration cross the first pixel wrap
    pk = synth.generate(synth.small(shot_begin=0, n_shots=560, pair_frac=0.05, dark_per_shot=2.0))[0]
    whole = oracle_run(pk)
    tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
    rng = np.random.default_rng(seed)
    cuts = [0] + sorted(rng.choice(tdc[1:], size=7, replace=False).tolist()) + [pk.size]
    labels, clusters, trig, state = run_calls(pk, cuts)
    assert np.array_equal(labels, whole["labels"])
    assert np.array_equal(trig, whole["triggers"])
    assert_clusters_equal(clusters, whole["clusters"])
    assert state["triggers"] == tdc.size
    assert state["pix_wraps"] == 1


def test_state_handed_to_another_context():
    pk = synth.generate(synth.small(shot_begin=0, n_shots=540))[0]
    whole = oracle_run(pk)
    tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
    cut = int(tdc[510])                       # after the first pixel wrap
    import torch
    a = tpx.Context(tpx.Config(), max_packets=pk.size)
    out = a.alloc_outputs(cut, True, False, cut, cut)
    a.tpx_process(to_device(pk[:cut]), out)
    a.tpx_sync()
    st = a.tpx_get_state()
    a.close()
    assert st["pix_wraps"] == 1 and st["triggers"] == 510
    b = tpx.Context(tpx.Config(), max_packets=pk.size)
    b.tpx_set_state(st)
    rest = pk[cut:]
    out = b.alloc_outputs(rest.size, True, False, rest.size, rest.size)
    b.tpx_process(to_device(rest), out, index_base=cut)
    rc, cnt = b.tpx_sync(check=False)
    r = b.collect(out, rc, cnt)
    b.close()
    assert rc == 0
    assert np.array_equal(r["labels"], whole["labels"][cut:])
    sel = whole["clusters"]["label"] >= cut
    assert_clusters_equal(r["clusters"], whole["clusters"][sel])
    assert np.array_equal(r["triggers"], whole["triggers"][510:])


def test_chained_general_path_redo():
    """The exact redo through the general path also continues the state."""
    rng = np.random.default_rng(5)
    from streams import StreamBuilder
    b = StreamBuilder()
    t0 = 7_000_000
    for s in range(3):
        b.tdc(t0 + s * 640_000)
        n = 9_000 if s == 1 else 300
        for _ in range(n):
            b.pix(rng.integers(0, 80), rng.integers(0, 80), rng.integers(1, 200), t0 + s * 640_000 + 900 + rng.integers(0, 3000))
    pk = b.packets()
    assert gpu_run(pk)["counters"]["redone"] == 1
    whole = oracle_run(pk)
    tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
    labels, clusters, trig, state = run_calls(pk, [0, int(tdc[1]), int(tdc[2]), pk.size])
    assert np.array_equal(labels, whole["labels"])
    assert_clusters_equal(clusters, whole["clusters"])
    assert state["triggers"] == 3


def test_shards_on_one_gpu_equal_one_call():
    """The multi-GPU shard pipeline, its ranks run one after another on one
    GPU: per-range unwrap summaries on the device, the in-order combination,
    and each range processed from its starting state."""
    from paper_2603_04942_gb300 import shard
    from test_shard_gloo import _summary
    pk = synth.generate(synth.small(shot_begin=350, n_shots=350, pair_frac=0.05))[0]
    whole = oracle_run(pk)
    cuts = shard.plan_cuts((pk >> np.uint64(60)) == 6, 3)
    summaries = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
        s = ctx.tpx_summarize(to_device(pk[a:b]))
        ctx.close()
        assert s == _summary(pk[a:b])
        summaries.append(s)
    states = shard.states_from_summaries(summaries)
    labels, clusters = [], []
    for (a, b), st in zip(zip(cuts[:-1], cuts[1:]), states):
        ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
        part = pk[a:b]
        out = ctx.alloc_outputs(part.size, True, False, part.size, part.size)
        shard.process_shard(ctx, to_device(part), a, st, out)
        rc, cnt = ctx.tpx_sync(check=False)
        assert rc == 0
        r = ctx.collect(out, rc, cnt)
        ctx.close()
        labels.append(r["labels"])
        clusters.append(r["clusters"])
    assert np.array_equal(np.concatenate(labels), whole["labels"])
    assert_clusters_equal(np.concatenate(clusters), whole["clusters"])


def test_shards_generated_apart_equal_one_call():
    """As the benchmark's ranks run: each shot range of one acquisition
    generated on its own (shots [r S, (r + 1) S)), its unwrap summary formed
    on the device, the summaries combined in rank order, each range processed
    from its starting state with its stream index base. Together they equal
    one oracle run over the whole acquisition (the pixel wrap at shot 500
    falls in the second range)."""
    from paper_2603_04942_gb300 import shard
    S, R = 400, 3
    whole = synth.generate(synth.large(n_shots=S * R))[0]
    parts = [synth.generate(synth.large(n_shots=S, shot_begin=r * S))[0] for r in range(R)]
    assert np.array_equal(np.concatenate(parts), whole)
    o = oracle_run(whole)
    summaries = []
    for pk in parts:
        ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
        summaries.append(ctx.tpx_summarize(to_device(pk)))
        ctx.close()
    states = shard.states_from_summaries(summaries)
    labels, clusters, trig = [], [], []
    base = 0
    for r, (pk, st) in enumerate(zip(parts, states)):
        ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
        if r > 0:
            ctx.tpx_set_state(st)
        out = ctx.alloc_outputs(pk.size, True, False, pk.size, pk.size)
        ctx.tpx_process(to_device(pk), out, index_base=base)
        rc, cnt = ctx.tpx_sync(check=False)
        assert rc == 0
        g = ctx.collect(out, rc, cnt)
        ctx.close()
        labels.append(g["labels"])
        clusters.append(g["clusters"])
        trig.append(g["triggers"])
        base += pk.size
    assert np.array_equal(np.concatenate(labels), o["labels"])
    assert np.array_equal(np.concatenate(trig), o["triggers"])
    assert_clusters_equal(np.concatenate(clusters), o["clusters"])


def test_kernel_timing_counts_each_fused_launch_and_leaves_results_unchanged():
    import torch
    pk = synth.generate(synth.small(shot_begin=0, n_shots=300, pair_frac=0.05))[0]
    ref = oracle_run(pk)
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        d = to_device(pk)
        ctx.tpx_kernel_timing(True)
        for _ in range(3):
            out = ctx.alloc_outputs(pk.size, True, False, pk.size, pk.size)
            ctx.tpx_process(d, out)
            rc, cnt = ctx.tpx_sync(check=False)
            assert rc == 0
        t = ctx.tpx_kernel_times()
        assert t["launches"] == 3
        assert t["fused_ms"] > 0 and t["prepass_ms"] > 0
        r = ctx.collect(out, rc, cnt)
        assert np.array_equal(r["labels"], ref["labels"])
        assert_clusters_equal(r["clusters"], ref["clusters"])
        # off: nothing more is recorded; on again: the sums restart
        ctx.tpx_kernel_timing(False)
        ctx.tpx_process(d, out)
        ctx.tpx_sync()
        assert ctx.tpx_kernel_times()["launches"] == 3
        ctx.tpx_kernel_timing(True)
        assert ctx.tpx_kernel_times()["launches"] == 0
        torch.cuda.synchronize()
    finally:
        ctx.close()
