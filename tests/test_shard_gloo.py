"""Multi-GPU shard logic on CPU ranks (gloo, world size 2): cut planning, the
one all_gather of unwrap summaries and their in-order combination. Each rank
then runs the oracle on its range from the exchanged state; the concatenated
records equal the single-stream run."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2603_04942_gb300 import shard

P_PIX, P_TDC = 1 << 34, 1 << 36


def _raws(pk):
    """Raw times of pixel and TDC packets (test-side restatement of the layout)."""
    hdr = pk >> np.uint64(60)
    w = pk.astype(np.uint64)
    coarse = ((w & np.uint64(0xFFFF)) << np.uint64(14)) | ((w >> np.uint64(30)) & np.uint64(0x3FFF))
    ftoa = (w >> np.uint64(16)) & np.uint64(0xF)
    praw = ((coarse.astype(np.int64) * 16 - ftoa.astype(np.int64)) % P_PIX)
    traw = ((((w >> np.uint64(9)) & np.uint64((1 << 35) - 1)).astype(np.int64)) * 2) % P_TDC
    return hdr == 0xB, praw, hdr == 0x6, traw


def _summary(pk):
    isp, praw, ist, traw = _raws(pk)
    out = {}
    for name, m, raw in (("pix", isp, praw), ("tdc", ist, traw)):
        v = raw[m]
        steps = np.diff(v)
        wraps = int(np.sum(steps < -shard.WRAP_THR_TICKS) - np.sum(steps > shard.WRAP_THR_TICKS))
        key = "pixels" if name == "pix" else "triggers"
        out[key] = int(v.size)
        out[f"{name}_first_raw"] = int(v[0]) if v.size else 0
        out[f"{name}_last_raw"] = int(v[-1]) if v.size else 0
        out[f"{name}_wraps"] = wraps
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    try:
        pk = synth.generate(synth.small(shot_begin=350, n_shots=350, pair_frac=0.05))[0]
        cuts = shard.plan_cuts((pk >> np.uint64(60)) == 6, world)
        a, b = cuts[rank], cuts[rank + 1]
        state, summaries = shard.exchange_states(_summary(pk[a:b]))
        np.save(os.path.join(outdir, f"state{rank}.npy"), np.array([state[f] for f in shard.STATE_FIELDS]))
        cfg = oracle.Config(epoch0_pix=state["pix_wraps"], epoch0_tdc=state["tdc_wraps"],
                            prev_pix_raw=state["pix_last_raw"] if state["pixels"] else None,
                            prev_tdc_raw=state["tdc_last_raw"] if state["triggers"] else None)
        r = oracle.run(pk[a:b], cfg, idx_base=a)
        cl = r["clusters"].copy()
        cl["shot"] += state["triggers"]
        gathered = [None] * world
        dist.all_gather_object(gathered, (cl, r["labels"], r["triggers"]))
        if rank == 0:
            np.save(os.path.join(outdir, "clusters.npy"), np.concatenate([g[0] for g in gathered]))
            np.save(os.path.join(outdir, "labels.npy"), np.concatenate([g[1] for g in gathered]))
            np.save(os.path.join(outdir, "triggers.npy"), np.concatenate([g[2] for g in gathered]))
            np.save(os.path.join(outdir, "cuts.npy"), np.array(cuts))
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_one_stream(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    pk = synth.generate(synth.small(shot_begin=350, n_shots=350, pair_frac=0.05))[0]
    full = oracle.run(pk, want_info=True)
    cuts = np.load(tmp_path / "cuts.npy")
    assert 0 < cuts[1] < pk.size and (pk[cuts[1]] >> np.uint64(60)) == 6
    # the exchanged starting state of rank 1 is the true state at its cut
    st = dict(zip(shard.STATE_FIELDS, np.load(tmp_path / "state1.npy").tolist()))
    info = full["info"]
    before = info[: cuts[1]]
    lp = np.flatnonzero(before["type"] == 1)[-1]
    lt = np.flatnonzero(before["type"] == 2)[-1]
    assert st["pixels"] == int((before["type"] == 1).sum())
    assert st["pix_wraps"] == int(before["t"][lp] // P_PIX) and st["pix_last_raw"] == int(before["t"][lp] % P_PIX)
    assert st["triggers"] == int((before["type"] == 2).sum())
    assert st["tdc_wraps"] == int(before["t"][lt] // P_TDC) and st["tdc_last_raw"] == int(before["t"][lt] % P_TDC)
    assert st["pix_wraps"] == 1            # rank 1 starts after the first pixel wrap
    # the concatenated shards equal the single stream
    assert np.array_equal(np.load(tmp_path / "labels.npy"), full["labels"])
    assert np.array_equal(np.load(tmp_path / "triggers.npy"), full["triggers"])
    cl = np.load(tmp_path / "clusters.npy")
    assert cl.size == full["clusters"].size
    for f in full["clusters"].dtype.names:
        assert np.array_equal(cl[f], full["clusters"][f]), f


def test_combine_is_associative_and_matches_whole():
    pk = synth.generate(synth.small(shot_begin=480, n_shots=60))[0]
    rng = np.random.default_rng(0)
    cuts = [0] + sorted(rng.choice(np.arange(1, pk.size), size=5, replace=False).tolist()) + [pk.size]
    parts = [_summary(pk[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    left = shard.identity()
    for p in parts:
        left = shard.combine(left, p)
    right = shard.identity()
    for p in reversed(parts):
        right = shard.combine(p, right)
    assert left == right == _summary(pk)


def _rank_dies(rank, world, port, outdir):
    """Rank 1 leaves between steps (after joining, before the exchange); rank
    0's exchange must end with an error within the group's timeout, not hang."""
    import datetime

    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)
    pk = synth.generate(synth.small(n_shots=40))[0]
    try:
        shard.exchange_states(_summary(pk))
        outcome = "completed"
    except Exception as e:   # the backend's error type differs between versions
        outcome = "error: " + type(e).__name__
    with open(os.path.join(outdir, "outcome.txt"), "w") as f:
        f.write(outcome)
    os._exit(0)   # the group is broken: leave without a collective teardown


def test_a_rank_that_dies_is_reported_by_the_exchange(tmp_path):
    import time

    import torch.multiprocessing as mp
    t0 = time.perf_counter()
    mp.spawn(_rank_dies, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    outcome = (tmp_path / "outcome.txt").read_text()
    assert outcome.startswith("error"), outcome
    assert time.perf_counter() - t0 < 120
