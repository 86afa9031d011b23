"""The fused kernel's second tile geometry (512-thread CTAs, two per SM,
2048-packet tiles, ranges of up to 4096 positions) against the oracle: the
same results as the default geometry, including ranges it cannot hold
(redone exactly by the general path) and chained calls."""
import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_parity, gpu_run, oracle_run, to_device
from streams import StreamBuilder, random_dense_stream

pytestmark = pytest.mark.gpu

T2 = 2048


@pytest.fixture(scope="module")
def small():
    return synth.generate(synth.small())


@pytest.mark.parametrize("mode", [0, 1])
def test_small_config(small, mode):
    pk = small[0] if mode == 0 else small[0][: 30 * T2 + 77]
    g, o = gpu_run(pk, mode=mode, tile=tpx.TILE_2048), oracle_run(pk, mode=mode)
    assert g["status"] == 0 and g["counters"]["redone"] == 0
    assert_parity(g, o)


def test_large_config_slice():
    pk = synth.generate(synth.large(n_shots=300))[0]
    g, o = gpu_run(pk, index_base=777, tile=tpx.TILE_2048), oracle_run(pk, index_base=777)
    assert g["status"] == 0
    assert_parity(g, o)


@pytest.mark.parametrize("n", [1, 5, T2 - 1, T2, T2 + 1, 3 * T2 + 11])
def test_ragged_sizes(small, n):
    pk = small[0][:n]
    g, o = gpu_run(pk, tile=tpx.TILE_2048), oracle_run(pk)
    assert g["status"] == 0
    assert_parity(g, o)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode", [0, 1])
def test_dense_random_streams(seed, mode):
    rng = np.random.default_rng(700 + seed)
    rx, ry, dt = [(1, 1, 32), (0, 2, 10), (2, 1, 0), (3, 3, 100)][seed]
    lut = rng.integers(-20, 20, size=1024).astype(np.int16) if seed % 2 else None
    pk = random_dense_stream(rng, n_shots=30, per_shot=140, area=7, t_spread=60).packets()
    g = gpu_run(pk, rx=rx, ry=ry, dt=dt, mode=mode, lut=lut, tile=tpx.TILE_2048)
    o = oracle_run(pk, rx=rx, ry=ry, dt=dt, mode=mode, lut=lut)
    assert g["status"] == 0
    assert_parity(g, o)


def test_shot_longer_than_the_smaller_range_is_redone():
    """A 5000-pixel shot fits the 8192-position ranges but not the 5120-position
    ones once its trigger's tile adds its own packets: the smaller geometry
    hands the call to the general path, exactly."""
    rng = np.random.default_rng(9)
    b = StreamBuilder()
    t = 20_000_000
    for s in range(4):
        b.tdc(t + s * 640_000)
        for _ in range(5000 if s == 1 else 200):
            b.pix(rng.integers(0, 256), rng.integers(0, 256), rng.integers(1, 200),
                  t + s * 640_000 + 900 + rng.integers(0, 40_000))
    pk = b.packets()
    g4 = gpu_run(pk)
    g2 = gpu_run(pk, tile=tpx.TILE_2048)
    o = oracle_run(pk)
    assert g4["counters"]["redone"] == 0 and g2["counters"]["redone"] == 1
    assert_parity(g4, o)
    assert_parity(g2, o)


def test_chained_calls():
    pk = synth.generate(synth.small(n_shots=540))[0]
    whole = oracle_run(pk)
    tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
    cuts = [0, int(tdc[101]), int(tdc[333]), int(tdc[512]), pk.size]
    ctx = tpx.Context(tpx.Config(chain=True, tile_geometry=tpx.TILE_2048), max_packets=pk.size)
    try:
        labels = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            out = ctx.alloc_outputs(b - a, True, False, b - a, b - a)
            ctx.tpx_process(to_device(pk[a:b]), out, index_base=a)
            rc, cnt = ctx.tpx_sync(check=False)
            assert rc == 0
            labels.append(ctx.collect(out, rc, cnt)["labels"])
        assert np.array_equal(np.concatenate(labels), whole["labels"])
    finally:
        ctx.close()


def _run_calls(pk, calls, cfg):
    ctx = tpx.Context(cfg, max_packets=pk.size)
    try:
        d = to_device(pk)
        outs = []
        for _ in range(calls):
            out = ctx.alloc_outputs(pk.size, True, False, pk.size, pk.size)
            ctx.tpx_process(d, out)
            rc, cnt = ctx.tpx_sync(check=False)
            assert rc == 0
            outs.append(ctx.collect(out, rc, cnt))
        return outs, ctx.tpx_tuning()
    finally:
        ctx.close()


def test_autotuner_times_both_geometries_and_keeps_one():
    pk = synth.generate(synth.small(n_shots=2300))[0]
    assert pk.size >= 1 << 20
    outs, tune = _run_calls(pk, 3, tpx.Config())
    assert tune["tile_geometry"] in (tpx.TILE_4096, tpx.TILE_2048)
    assert tune["ms_per_mpacket"]["4096"] > 0 and tune["ms_per_mpacket"]["2048"] > 0
    o = oracle_run(pk)
    for g in outs:
        assert_parity(g, o)


def test_autotuner_avoids_the_geometry_that_needed_a_redo():
    """3500-pixel shots fit every 8192-position range (at most 4095 + 3501
    positions) but overflow many 5120-position ones: the sample on the
    2048-packet tiles is redone by the general path and loses."""
    rng = np.random.default_rng(13)
    b = StreamBuilder()
    t = 30_000_000
    for s in range(310):
        b.tdc(t + s * 640_000)
        for _ in range(3500):
            b.pix(rng.integers(0, 256), rng.integers(0, 256), rng.integers(1, 300),
                  t + s * 640_000 + 900 + rng.integers(0, 60_000))
    pk = b.packets()
    outs, tune = _run_calls(pk, 3, tpx.Config())
    assert outs[0]["counters"]["redone"] == 1 and outs[1]["counters"]["redone"] == 0
    assert tune["tile_geometry"] == tpx.TILE_4096
    assert outs[2]["counters"]["redone"] == 0
    o = oracle_run(pk)
    for g in outs:
        assert_parity(g, o)


def test_explicit_geometry_is_not_tuned():
    pk = synth.generate(synth.small(n_shots=2300))[0]
    _, tune = _run_calls(pk, 1, tpx.Config(tile_geometry=tpx.TILE_4096))
    assert tune["tile_geometry"] == tpx.TILE_4096
    assert tune["ms_per_mpacket"]["2048"] == 0
