"""GPU parity of the general path: tpx_decode -> tpx_cluster -> tpx_centroid
(global memory, radix sort on ToA, no range limit) against the oracle, and the
exact redo of tpx_process calls whose input the fused kernel cannot hold."""
import numpy as np
import pytest

import oracle
import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_clusters_equal, assert_parity, gpu_run, oracle_run, to_device
from streams import StreamBuilder, random_dense_stream

pytestmark = pytest.mark.gpu


def unfused(pk, *, rx=1, ry=1, dt=32, mode=0, tof_max=64_000, lut=None, index_base=0):
    import torch
    dlut = None if lut is None else torch.from_numpy(np.asarray(lut, np.int16)).cuda()
    ctx = tpx.Context(tpx.Config(rx=rx, ry=ry, dt_ticks=dt, mode=mode, tof_max_ticks=tof_max, timewalk_lut=dlut),
                      max_packets=max(1, pk.size))
    try:
        d = to_device(pk) if pk.size else torch.zeros(2, dtype=torch.int64, device="cuda")
        dec = ctx.tpx_decode(d, index_base=index_base, n_packets=pk.size)
        rc_dec, cnt = ctx.tpx_sync(check=False)
        nh = int(dec["n_hits"].item())
        cl = ctx.tpx_cluster(dec["hits"], nh)
        ce = ctx.tpx_centroid(dec["hits"], cl["labels"], cl["is_peak"], nh)
        rc, cnt2 = ctx.tpx_sync(check=False)
        ncl = int(ce["n_clusters"].item())
        raw = ce["clusters"][: ncl * tpx.CLUSTER_DTYPE.itemsize].cpu().numpy()
        h = {k: v[:nh].cpu().numpy() for k, v in dec["hits"].items()}
        # per-packet labels from per-hit labels
        labels = np.full(pk.size, -1, np.int64)
        peaks = np.zeros(pk.size, np.uint8)
        labels[h["index"] - index_base] = cl["labels"][:nh].cpu().numpy()
        peaks[h["index"] - index_base] = cl["is_peak"][:nh].cpu().numpy()
        return dict(status=rc_dec or rc, hits=h, n_hits=nh, labels=labels, is_peak=peaks,
                    clusters=np.frombuffer(raw.tobytes(), tpx.CLUSTER_DTYPE).copy(), n_clusters=ncl,
                    triggers=dec["trig"][: int(dec["n_trig"].item())].cpu().numpy(), counters=cnt)
    finally:
        ctx.close()


def check_unfused(pk, **kw):
    g = unfused(pk, **kw)
    o = oracle_run(pk, **kw)
    assert g["status"] == 0
    assert np.array_equal(g["triggers"], o["triggers"])
    assert np.array_equal(g["labels"], o["labels"])
    assert np.array_equal(g["is_peak"], o["is_peak"])
    assert g["n_clusters"] == o["clusters"].size
    assert_clusters_equal(g["clusters"], o["clusters"])
    return g, o


def test_unfused_small_config():
    pk = synth.generate(synth.small(n_shots=300, pair_frac=0.05, dark_per_shot=3.0))[0]
    g, o = check_unfused(pk, index_base=99)
    # decode view: kept pixels, their shots and corrected times
    info = oracle.run(pk, want_info=True)["info"]
    kept = np.flatnonzero(o["labels"] >= 0)
    assert np.array_equal(g["hits"]["index"], kept + 99)
    assert np.array_equal(g["hits"]["shot"], info["shot"][kept])
    assert np.array_equal(g["hits"]["t"], info["t"][kept])
    assert np.array_equal(g["hits"]["x"], info["x"][kept])
    assert np.array_equal(g["hits"]["tot"].astype(np.int64), info["tot"][kept])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_unfused_dense_random(mode, seed):
    rng = np.random.default_rng(900 + seed)
    rx, ry, dt = [(1, 1, 32), (0, 2, 10), (2, 1, 0), (3, 3, 100)][seed]
    lut = rng.integers(-20, 20, size=1024).astype(np.int16) if seed % 2 else None
    pk = random_dense_stream(rng, n_shots=30, per_shot=200, area=8, t_spread=60).packets()
    check_unfused(pk, rx=rx, ry=ry, dt=dt, mode=mode, lut=lut)


@pytest.mark.parametrize("mode", [0, 1])
def test_unfused_segments_longer_than_a_warp_buffer(mode):
    """Hits closer than dt chain into time segments of several hundred hits:
    beyond one warp's shared buffer, so the global-memory kernels take them,
    next to short segments in the same call."""
    rng = np.random.default_rng(31 + mode)
    pk = random_dense_stream(rng, n_shots=12, per_shot=700, area=10, t_spread=80).packets()
    check_unfused(pk, mode=mode, dt=4)
    check_unfused(pk, mode=mode, dt=40)


def test_unfused_large_slice():
    pk = synth.generate(synth.large(n_shots=150))[0]
    check_unfused(pk)


def test_fallback_for_a_shot_longer_than_the_range():
    """A 10,000-pixel shot exceeds the fused kernel's 8192-position range:
    tpx_sync redoes the call with the general path, exactly."""
    rng = np.random.default_rng(17)
    b = StreamBuilder()
    t0 = 5_000_000
    b.tdc(t0)
    for _ in range(10_000):
        b.pix(rng.integers(0, 64), rng.integers(0, 64), rng.integers(1, 300), t0 + 700 + rng.integers(0, 3000))
    b.tdc(t0 + 640_000)
    for _ in range(500):
        b.pix(rng.integers(0, 256), rng.integers(0, 256), 40, t0 + 640_000 + 900 + rng.integers(0, 100))
    pk = b.packets()
    g, o = gpu_run(pk), oracle_run(pk)
    assert g["status"] == 0 and g["counters"]["redone"] == 1
    assert_parity(g, o)


def test_fallback_for_pixels_whose_trigger_is_outside_the_range():
    """Triggers closer together than the ToF cut and pixels reported after the
    next trigger's packet: the fused kernel cannot bin them inside its range."""
    rng = np.random.default_rng(23)
    b = StreamBuilder()
    period = 20_000
    for s in range(40):
        tt = 10_000_000 + s * period
        b.tdc(tt)
        ev = [(rng.integers(0, 32), rng.integers(0, 32), rng.integers(1, 100), tt + rng.integers(0, 30_000))
              for _ in range(60)]
        for e in ev:
            b.pix(*e)
    pk = b.packets()
    g, o = gpu_run(pk), oracle_run(pk)
    assert g["status"] == 0 and g["counters"]["redone"] == 1
    assert_parity(g, o)
    gp, op = gpu_run(pk, mode=1), oracle_run(pk, mode=1)
    assert gp["counters"]["redone"] == 1
    assert_parity(gp, op)


def test_normal_input_is_not_redone():
    pk = synth.generate(synth.small(n_shots=50))[0]
    assert gpu_run(pk)["counters"]["redone"] == 0


def test_an_unsynchronised_call_that_needed_the_general_path_is_reported():
    """Only the last call before tpx_sync is redone; when an earlier call
    needed it, tpx_sync reports TPX_EUNSUPPORTED instead of returning that
    call's incomplete outputs as if they were fine."""
    rng = np.random.default_rng(41)
    b = StreamBuilder()
    t0 = 5_000_000
    b.tdc(t0)
    for _ in range(10_000):   # longer than any range
        b.pix(rng.integers(0, 64), rng.integers(0, 64), rng.integers(1, 300), t0 + 700 + rng.integers(0, 3000))
    b.tdc(t0 + 640_000)
    long_pk = b.packets()
    ok_pk = synth.generate(synth.small(n_shots=40))[0]
    ctx = tpx.Context(tpx.Config(tile_geometry=tpx.TILE_4096), max_packets=max(long_pk.size, ok_pk.size))
    try:
        d_long, d_ok = to_device(long_pk), to_device(ok_pk)
        out1 = ctx.alloc_outputs(long_pk.size, True, False, long_pk.size, 16)
        out2 = ctx.alloc_outputs(ok_pk.size, True, False, ok_pk.size, 64)
        ctx.tpx_process(d_long, out1)
        ctx.tpx_process(d_ok, out2)
        rc, _ = ctx.tpx_sync(check=False)
        assert rc == -9   # TPX_EUNSUPPORTED
        # synchronised calls are exact again
        ctx.tpx_process(d_long, out1)
        rc, cnt = ctx.tpx_sync(check=False)
        assert rc == 0 and cnt["redone"] == 1
        assert_parity(ctx.collect(out1, rc, cnt), oracle_run(long_pk), check_counters=False)
    finally:
        ctx.close()
