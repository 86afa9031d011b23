"""GPU parity: the fused CUDA path against the CPU oracle on the same seeded
inputs, bit-exact on labels, peaks, triggers and integer cluster fields,
within 1e-6 on the final divisions. Sizes span many tiles (4096 packets) and
ragged tails; edge cases cover empty input, missing triggers, corrupt
packets, pixel-wrap stragglers, long triggerless stretches and both modes."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_parity, gpu_run, oracle_run
from streams import StreamBuilder, random_dense_stream

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.fixture(scope="module")
def small():
    return synth.generate(synth.small())


def test_small_config_full(small):
    pk, truth, trig = small
    g = gpu_run(pk)
    o = oracle_run(pk)
    assert g["status"] == 0 and o["status"] == 0
    assert_parity(g, o)
    assert np.array_equal(g["triggers"], trig)


def test_small_config_paper_mode(small):
    pk = small[0][: 60 * TILE + 123]
    g = gpu_run(pk, mode=1)
    o = oracle_run(pk, mode=1)
    assert g["status"] == 0
    assert_parity(g, o)


def test_pairs_dark_counts_and_stated_size():
    for p in (synth.small(n_shots=300, pair_frac=0.05, dark_per_shot=4.0, seed=11),
              synth.stated_size(synth.small(n_shots=300, seed=12, pair_frac=0.05))):
        pk = synth.generate(p)[0]
        g, o = gpu_run(pk), oracle_run(pk)
        assert g["status"] == 0
        assert_parity(g, o)


def test_large_config_slice_with_index_base():
    """A slice of the large configuration (Poisson 50, pairs) at an index base."""
    pk = synth.generate(synth.large(n_shots=400))[0]
    g = gpu_run(pk, index_base=123_456_789)
    o = oracle_run(pk, index_base=123_456_789)
    assert_parity(g, o)


@pytest.mark.parametrize("n", [1, 2, 3, 17, TILE - 1, TILE, TILE + 1, 2 * TILE + 7, 5 * TILE - 3])
def test_ragged_sizes(small, n):
    pk = small[0][:n]
    g, o = gpu_run(pk), oracle_run(pk)
    assert g["status"] == 0
    assert_parity(g, o)


@pytest.mark.parametrize("start", [1, 5, TILE - 2, TILE + 333])
def test_stream_starting_mid_shot(small, start):
    """Pixels before the first trigger of the call are dropped (no trigger
    precedes them), possibly across several tiles."""
    pk = small[0][start: start + 6 * TILE]
    g, o = gpu_run(pk), oracle_run(pk)
    assert_parity(g, o)


def test_empty_and_triggerless():
    g = gpu_run(np.zeros(0, np.uint64))
    assert g["status"] == 0 and g["n_clusters"] == 0 and g["n_trig"] == 0
    b = StreamBuilder()
    for i in range(3 * TILE + 5):
        b.pix(i % 256, (i * 7) % 256, 20, 1000 + i)
    pk = b.packets()
    g, o = gpu_run(pk), oracle_run(pk)
    assert_parity(g, o)
    assert g["counters"]["dropped_pre_trigger"] == pk.size


def test_shot_spanning_tiles_and_tdc_only_tiles():
    """A long shot crossing a tile boundary (the owner reads ahead), tiles
    holding only TDC packets, and a stream ending without a terminating TDC."""
    b = StreamBuilder()
    rng = np.random.default_rng(5)
    t = 10_000_000
    for s in range(3):
        b.tdc(t + s * 640_000)
        for i in range(3000 + 500 * s):
            b.pix(rng.integers(0, 256), rng.integers(0, 256), rng.integers(1, 100),
                  t + s * 640_000 + 1000 + rng.integers(0, 60_000))
    for s in range(3, 3 + 2 * TILE):       # many empty shots
        b.tdc(t + s * 640_000)
    s = 3 + 2 * TILE
    b.tdc(t + s * 640_000)
    for i in range(900):
        b.pix(rng.integers(0, 256), rng.integers(0, 256), 50, t + s * 640_000 + 500 + i)
    pk = b.packets()
    g, o = gpu_run(pk), oracle_run(pk)
    assert g["status"] == 0
    assert_parity(g, o)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("mode", [0, 1])
def test_dense_random_streams(seed, mode):
    rng = np.random.default_rng(500 + seed)
    rx, ry, dt = [(1, 1, 32), (0, 2, 10), (2, 1, 0), (3, 3, 100)][seed % 4]
    lut = rng.integers(-20, 20, size=1024).astype(np.int16) if seed % 2 else None
    b = random_dense_stream(rng, n_shots=40, per_shot=150 + 10 * seed, area=6 + seed, t_spread=60)
    pk = b.packets()
    g = gpu_run(pk, rx=rx, ry=ry, dt=dt, mode=mode, lut=lut, index_base=seed * 1000)
    o = oracle_run(pk, rx=rx, ry=ry, dt=dt, mode=mode, lut=lut, index_base=seed * 1000)
    assert g["status"] == 0
    assert_parity(g, o)


@pytest.mark.parametrize("mode", [0, 1])
def test_large_box_radius(small, mode):
    """A 5-pixel box radius (the size of the paper's toy neighbourhood,
    Sec. V.A) on a slice of the small configuration: many more cells per
    hit, partners beyond eight per pixel (the serial union fallback)."""
    pk = small[0][: 25 * TILE + 11]
    g = gpu_run(pk, rx=5, ry=5, dt=100, mode=mode)
    o = oracle_run(pk, rx=5, ry=5, dt=100, mode=mode)
    assert g["status"] == 0
    assert_parity(g, o)


def test_pixel_wrap_straddle_and_stragglers(small):
    """Shot 500 of the small configuration straddles the 2^34-tick pixel wrap
    with pre-wrap pixels reported after post-wrap ones (Sec. IV.A)."""
    pk = synth.generate(synth.small(shot_begin=0, n_shots=520))[0]
    tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
    sl = pk[tdc[495]:]
    # slice starts after no wrap (epoch 0), so the oracle needs no initial epochs
    g, o = gpu_run(sl), oracle_run(sl)
    assert_parity(g, o)
    # the straddling shot has clusters with pixels on both sides of the wrap
    ct = g["clusters"][g["clusters"]["shot"] == 5]
    assert ct.size > 10


def test_corrupt_packets_and_strict_mode(small):
    pk = small[0][: 3 * TILE].copy()
    pk[[7, 100, 5000, 9000]] = np.uint64(0x1234_5678_9ABC_DEF0)
    g, o = gpu_run(pk), oracle_run(pk)
    assert g["status"] == 0 and g["counters"]["corrupt"] == 4
    assert_parity(g, o)
    gs = gpu_run(pk, strict=True)
    assert gs["status"] == -4 and oracle_run(pk, strict=True)["status"] == -4


def test_decreasing_triggers_flagged():
    b = StreamBuilder()
    b.tdc(5_000_000)
    b.pix(1, 1, 10, 5_000_100)
    b.tdc(4_000_000)
    b.pix(2, 2, 10, 4_000_100)
    pk = b.packets()
    assert gpu_run(pk)["status"] == -4
    assert oracle_run(pk)["status"] == -4


def test_output_capacity_overflow_reports_required_count(small):
    pk = small[0][: 10 * TILE]
    o = oracle_run(pk)
    g = gpu_run(pk, cluster_capacity=100)
    assert g["status"] == -3 and g["n_clusters"] == o["clusters"].size
    assert np.array_equal(g["clusters"], o["clusters"][:100].astype(g["clusters"].dtype)) or \
        (g["clusters"]["label"] == o["clusters"]["label"][:100]).all()


def test_deterministic_repeat(small):
    pk = small[0]
    a, b = gpu_run(pk), gpu_run(pk)
    assert np.array_equal(a["labels"], b["labels"])
    assert a["clusters"].tobytes() == b["clusters"].tobytes()
