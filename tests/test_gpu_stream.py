"""Streaming: chunks of any size in, records of closed shots out. The union
of all chunks' records equals the single-stream result (oracle), including a
high-rate stream whose ToF cut spans the whole trigger period (pixels of a
shot are read out after the next trigger); streams give the same results alone
and run concurrently; admission answers EAGAIN; a stream checkpointed to a
host block and restored into a new stream continues exactly."""
import threading

import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import INT_FIELDS, assert_clusters_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def run_stream(pk, chunk_sizes, cfg=None, hold=2, max_chunk=None, slots=2, cuda_stream=None):
    st = tpx.Stream(cfg or tpx.Config(), max_chunk_packets=max_chunk or max(chunk_sizes), max_hold_packets=1 << 20,
                    hold_triggers=hold, slots=slots, stream=cuda_stream)
    try:
        recs, trig, first = [], [], []
        pos = 0
        for c in chunk_sizes:
            t = st.submit(pk[pos:pos + c])
            r = st.poll(t)
            assert r["status"] == 0
            recs.append(r["clusters"])
            trig.append(r["triggers"])
            first.append(r["first_shot"])
            pos += c
        assert pos == pk.size
        r = st.poll(st.finish())
        recs.append(r["clusters"])
        trig.append(r["triggers"])
        return np.concatenate(recs), np.concatenate(trig), first
    finally:
        st.close()


def chunks_for(n, rng, lo, hi):
    sizes = []
    while sum(sizes) < n:
        sizes.append(int(min(rng.integers(lo, hi), n - sum(sizes))))
    return sizes


def test_stream_small_config_in_random_chunks():
    pk = synth.generate(synth.small(n_shots=400, pair_frac=0.05))[0]
    whole = oracle_run(pk)
    rng = np.random.default_rng(1)
    recs, trig, first = run_stream(pk, chunks_for(pk.size, rng, 1, 30_000))
    assert np.array_equal(trig, whole["triggers"])
    assert_clusters_equal(recs, whole["clusters"])
    assert all(b >= a for a, b in zip(first, first[1:]))


def test_stream_several_chunks_in_flight_equal_the_oracle():
    """Up to `slots` chunks are submitted before any result is polled; each
    ticket's records come back in submission order and their union is the
    oracle's result over the whole stream."""
    pk = synth.generate(synth.small(n_shots=400, pair_frac=0.05))[0]
    whole = oracle_run(pk)
    rng = np.random.default_rng(7)
    sizes = chunks_for(pk.size, rng, 1, 20_000)
    st = tpx.Stream(tpx.Config(), max_chunk_packets=max(sizes), max_hold_packets=1 << 20, hold_triggers=2, slots=4)
    try:
        recs, trig, pos, i = [], [], 0, 0
        while i < len(sizes):
            tickets = []
            for c in sizes[i:i + 4]:
                tickets.append(st.submit(pk[pos:pos + c]))
                pos += c
            i += len(tickets)
            for t in tickets:
                r = st.poll(t)
                assert r["status"] == 0
                recs.append(r["clusters"])
                trig.append(r["triggers"])
        r = st.poll(st.finish())
        recs.append(r["clusters"])
        trig.append(r["triggers"])
    finally:
        st.close()
    assert np.array_equal(np.concatenate(trig), whole["triggers"])
    assert_clusters_equal(np.concatenate(recs), whole["clusters"])


def test_stream_high_rate_full_period():
    """10 Mhit/s ion-like stream, ToF cut = the whole period: shots hold ~10k
    pixels and their late pixels follow the next trigger packet."""
    p = synth.streaming(10e6, 30)
    pk = synth.generate(p)[0]
    tofm = synth.STREAM_TOF_MAX_TICKS
    o = oracle_run(pk, tof_max=tofm)
    assert o["status"] == 0 and o["clusters"].size > 5000
    rng = np.random.default_rng(2)
    recs, trig, _ = run_stream(pk, chunks_for(pk.size, rng, 5_000, 60_000), cfg=tpx.Config(tof_max_ticks=tofm))
    assert np.array_equal(trig, o["triggers"])
    # a late cluster of shot k can carry a larger label than an early cluster
    # of shot k+1 but is emitted with shot k: compare in label order
    assert_clusters_equal(np.sort(recs, order="label"), o["clusters"])


def test_streams_alone_and_concurrent_agree():
    import torch
    pks = [synth.generate(synth.small(n_shots=200, seed=40 + i))[0] for i in range(3)]
    sizes = [chunks_for(pk.size, np.random.default_rng(i), 2_000, 20_000) for i, pk in enumerate(pks)]
    alone = [run_stream(pk, sz)[0] for pk, sz in zip(pks, sizes)]
    out = [None] * 3
    errs = []

    def worker(i):
        try:
            out[i] = run_stream(pks[i], sizes[i], cuda_stream=torch.cuda.Stream())[0]
        except Exception as e:   # surfaced below
            errs.append(e)
    th = [threading.Thread(target=worker, args=(i,)) for i in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for a, b in zip(alone, out):
        assert a.size == b.size
        for f in INT_FIELDS:
            assert np.array_equal(a[f], b[f])


def test_admission():
    pk = synth.generate(synth.small(n_shots=20))[0]
    st = tpx.Stream(tpx.Config(), max_chunk_packets=pk.size, max_hold_packets=1 << 16, slots=1)
    t = st.submit(pk[:5000])
    with pytest.raises(tpx.TpxError) as e:
        st.submit(pk[5000:])
    assert e.value.code == tpx.EAGAIN
    st.poll(t)
    st.poll(st.submit(pk[5000:]))
    st.close()
    with pytest.raises(tpx.TpxError) as e:   # its buffers alone exceed a 1 MB budget
        tpx.Stream(tpx.Config(), max_chunk_packets=1 << 16, max_hold_packets=1 << 16, hbm_budget_bytes=1 << 20)
    assert e.value.code == tpx.EAGAIN


@pytest.mark.parametrize("kind", ["small", "high_rate"])
def test_checkpoint_and_resume_continue_the_stream_exactly(kind):
    """Halfway through, the stream's carry goes to a host block, the stream
    is destroyed, and a new stream restored from the block takes the rest:
    the records and triggers equal one uninterrupted run."""
    if kind == "small":
        pk = synth.generate(synth.small(n_shots=400, pair_frac=0.05))[0]
        cfg = tpx.Config()
        whole = oracle_run(pk)
    else:
        pk = synth.generate(synth.streaming(10e6, n_shots=60))[0]
        cfg = tpx.Config(tof_max_ticks=synth.STREAM_TOF_MAX_TICKS)
        whole = oracle_run(pk, tof_max=synth.STREAM_TOF_MAX_TICKS)
    sizes = chunks_for(pk.size, np.random.default_rng(5), 1000, 40_000)
    half = len(sizes) // 2
    kw = dict(max_chunk_packets=max(sizes), max_hold_packets=1 << 20, hold_triggers=2, slots=2)
    recs, trig, pos = [], [], 0
    st = tpx.Stream(cfg, **kw)
    for c in sizes[:half]:
        r = st.poll(st.submit(pk[pos:pos + c]))
        recs.append(r["clusters"])
        trig.append(r["triggers"])
        pos += c
    block = st.snapshot()
    with pytest.raises(tpx.TpxError) as e:
        st.restore(block)                  # a stream already in use
    assert e.value.code == tpx.EINVAL
    st.close()
    other = tpx.Stream(tpx.Config(dt_ticks=cfg.dt_ticks + 1, tof_max_ticks=cfg.tof_max_ticks), **kw)
    with pytest.raises(tpx.TpxError):
        other.restore(block)               # another configuration
    other.close()
    st = tpx.Stream(cfg, **kw)
    try:
        with pytest.raises(tpx.TpxError):
            st.restore(block[:-8] if len(block) > 8 else b"")   # a damaged block
        st.restore(block)
        for c in sizes[half:]:
            r = st.poll(st.submit(pk[pos:pos + c]))
            recs.append(r["clusters"])
            trig.append(r["triggers"])
            pos += c
        r = st.poll(st.finish())
        recs.append(r["clusters"])
        trig.append(r["triggers"])
    finally:
        st.close()
    assert np.array_equal(np.concatenate(trig), whole["triggers"])
    # results come in shot order; a late cluster of shot k can carry a larger
    # label than an early one of shot k+1: compare in label order
    assert_clusters_equal(np.sort(np.concatenate(recs), order="label"), whole["clusters"])
