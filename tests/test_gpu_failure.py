"""Failure detection on the GPU without a fault: a tile whose look-back
flags stay unpublished (tpx_debug_hold_tile) makes its successors' bounded
waits run out; the call completes, tpx_sync reports TPX_EDEVTIMEOUT, and the
same context then processes the next call exactly."""
import time

import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_parity, oracle_run, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile", [1, 40])
def test_device_wait_timeout_is_reported_and_the_context_recovers(tile):
    pk = synth.generate(synth.small())[0]          # ~5e5 packets: ~120 tiles of 4096
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        d = to_device(pk)
        ctx.tpx_debug_hold_tile(tile)
        out = ctx.alloc_outputs(pk.size, labels=True)
        t0 = time.perf_counter()
        ctx.tpx_process(d, out)
        rc, counters = ctx.tpx_sync(check=False)
        assert rc == tpx.EDEVTIMEOUT
        assert counters["redone"] == 0                # a timed-out call is not redone
        assert time.perf_counter() - t0 < 20          # one bounded wait, then the others give up
        g = ctx.process(d, labels=True, is_peak=True, check=False)
        assert g["status"] == 0
        assert_parity(g, oracle_run(pk))
        # a hold applies to one call only
        g2 = ctx.process(d, labels=True, is_peak=True, check=False)
        assert g2["status"] == 0 and np.array_equal(g2["labels"], g["labels"])
    finally:
        ctx.close()
