"""GPU-vs-oracle parity at the size the benchmark runs its kernel: more than
2^24 packets of the large-batch recipe (Poisson(50) particles per shot, 5%
overlapping pairs), placed across the first TDC wrap (2^36 ticks, shot 81,031
of the recipe's time line), where a pixel wrap (2^34 ticks) falls as well
(Sec. IV.A: both streams wrap, each unwrapped on its own).

Both sides start from the wrap counts at the slice start (three pixel
wraps, no TDC wrap yet: without them the pixel and TDC clocks of a slice from
the middle of an acquisition disagree and no pixel has a trigger), so the
slice computes what the whole acquisition would. One context runs the call
three times with the default tile geometry: the autotuner times both
geometries on the first two calls (each at least 2^20 packets) and keeps one
for the third; every call's labels, local-maximum flags, triggers, records and
counters equal the oracle's, bit for bit (centroids within 1e-6)."""
import numpy as np
import pytest

import oracle
import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_parity, to_device

pytestmark = pytest.mark.gpu

FIRST_TDC_WRAP_SHOT = 81_031      # first trigger at or after 2^36 ticks on the recipe's time line
N_SHOTS = 13_400                  # ~1.7e7 packets > 2^24


def _slice():
    p = synth.large(shot_begin=FIRST_TDC_WRAP_SHOT - N_SHOTS // 2, n_shots=N_SHOTS)
    st = synth.Stream(p)
    pk = st.packets()
    wraps = st.wrap_counts()
    st.close()
    trig_t = p.t_start_ticks + (p.shot_begin + np.arange(N_SHOTS, dtype=np.int64)) * p.trig_period_ticks
    assert trig_t[0] < synth.TDC_PERIOD_TICKS <= trig_t[-1], "the slice crosses the TDC wrap"
    assert pk.size > (1 << 24)
    return pk, wraps


@pytest.fixture(scope="module")
def scale_slice():
    return _slice()


def _run(ctx, d, n, wraps, index_base=0):
    e_pix, e_tdc = wraps
    ctx.tpx_set_state(dict(pixels=0, pix_last_raw=0, pix_wraps=e_pix, triggers=0, tdc_last_raw=0,
                           tdc_wraps=e_tdc))
    out = ctx.alloc_outputs(n, True, True, n // 8, N_SHOTS + 16)
    ctx.tpx_process(d, out, index_base)
    rc, counters = ctx.tpx_sync(check=False)
    return ctx.collect(out, rc, counters)


def _oracle(pk, wraps, index_base=0):
    o = oracle.run(pk, oracle.Config(epoch0_pix=wraps[0], epoch0_tdc=wraps[1]), idx_base=index_base)
    assert o["status"] == 0
    # inside the slice the TDC stream wraps: raw times restart below 2^36,
    # the unwrapped ones run past it; almost every pixel is kept
    assert o["triggers"][0] < synth.TDC_PERIOD_TICKS <= o["triggers"][-1]
    assert o["counters"]["kept"] > 0.99 * o["counters"]["pixels"]
    return o


def test_large_recipe_across_the_tdc_wrap_autotuned(scale_slice):
    pk, wraps = scale_slice
    o = _oracle(pk, wraps, index_base=3)
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        d = to_device(pk)
        geos = []
        for _ in range(3):
            g = _run(ctx, d, pk.size, wraps, index_base=3)
            assert g["status"] == 0
            assert g["counters"]["redone"] == 0
            assert_parity(g, o)
            geos.append(ctx.tpx_tuning())
        tune = geos[-1]
        # both geometries were timed, one was kept
        assert tune["tile_geometry"] in (tpx.TILE_4096, tpx.TILE_2048)
        assert tune["ms_per_mpacket"]["4096"] > 0 and tune["ms_per_mpacket"]["2048"] > 0
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", [tpx.MODE_CC, tpx.MODE_PAPER])
def test_large_recipe_across_the_tdc_wrap_4096_tiles(scale_slice, mode):
    pk, wraps = scale_slice
    o = oracle.run(pk, oracle.Config(epoch0_pix=wraps[0], epoch0_tdc=wraps[1], mode=mode))
    assert o["status"] == 0
    ctx = tpx.Context(tpx.Config(tile_geometry=tpx.TILE_4096, mode=mode), max_packets=pk.size)
    try:
        g = _run(ctx, to_device(pk), pk.size, wraps)
        assert g["status"] == 0 and g["counters"]["redone"] == 0
        assert_parity(g, o)
    finally:
        ctx.close()
