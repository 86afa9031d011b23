"""64-byte records (TPX_FLAG_RECORDS64): every record equals the first 64
bytes of the full record on every path that writes them -- the fused kernel
(CC and PAPER modes), the general-path redo of tpx_sync, the pipelined and
host-direct host calls -- and the derived x, y, ToF follow from the exact
sums. A batch call with the flag is rejected. The allocation-free entry
point's 64-byte records are tested with its other tests."""
import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import oracle_run, to_device

pytestmark = pytest.mark.gpu

FIELDS = tpx.CLUSTER64_DTYPE.names


def _same(r64: np.ndarray, full: np.ndarray):
    assert r64.dtype == tpx.CLUSTER64_DTYPE
    assert r64.size == full.size
    for f in FIELDS:
        assert np.array_equal(r64[f], full[f]), f


def _device(pk, cfg, **kw):
    ctx = tpx.Context(cfg, max_packets=pk.size)
    try:
        return ctx.process(to_device(pk), labels=True, is_peak=True, check=False, **kw)
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", [tpx.MODE_CC, tpx.MODE_PAPER])
def test_device_call_records64_equal_the_oracle(mode):
    pk = synth.generate(synth.small(shot_begin=0, n_shots=600, pair_frac=0.05, dark_per_shot=2.0))[0]
    ref = oracle_run(pk, mode=mode)
    r = _device(pk, tpx.Config(mode=mode, records64=True))
    assert r["status"] == 0
    _same(r["clusters"], ref["clusters"])
    assert np.array_equal(r["labels"], ref["labels"])
    # the derived centroid from the exact sums
    c = r["clusters"]
    np.testing.assert_allclose(c["s_x"] / c["s_tot"], ref["clusters"]["x"], rtol=0, atol=1e-12)


def test_redo_writes_records64():
    pk = synth.generate(synth.streaming(10e6, n_shots=40))[0]
    cfg = dict(tof_max_ticks=synth.STREAM_TOF_MAX_TICKS)
    ref = oracle_run(pk, tof_max=synth.STREAM_TOF_MAX_TICKS)
    r = _device(pk, tpx.Config(records64=True, **cfg), cluster_capacity=pk.size, trig_capacity=pk.size)
    assert r["status"] == 0 and r["counters"]["redone"] == 1
    _same(r["clusters"], ref["clusters"])


@pytest.mark.parametrize("direct", [False, True])
def test_host_call_records64_equal_full_records(direct):
    import torch
    pk = synth.generate(synth.large(n_shots=14_000))[0]
    assert pk.size >= 1 << 24   # pipelined when staged
    out = {}
    for r64 in (False, True):
        dt = tpx.CLUSTER64_DTYPE if r64 else tpx.CLUSTER_DTYPE
        ctx = tpx.Context(tpx.Config(records64=r64, labels32=True, host_direct=direct), max_packets=pk.size)
        try:
            n_cl = pk.size // 8
            if direct:
                hp = torch.from_numpy(pk.view(np.int64)).pin_memory()
                lab_t = torch.empty(pk.size, dtype=torch.int32, pin_memory=True)
                cl_t = torch.empty(n_cl * dt.itemsize, dtype=torch.uint8, pin_memory=True)
                tr_t = torch.empty(pk.size // 8, dtype=torch.int64, pin_memory=True)
                src, lab, cl, tr = hp.numpy().view(np.uint64), lab_t.numpy(), cl_t.numpy().view(dt), tr_t.numpy()
            else:
                src, lab = pk, np.empty(pk.size, np.int32)
                cl, tr = np.empty(n_cl, dt), np.empty(pk.size // 8, np.int64)
            rc, ncl, ntr = ctx.tpx_process_host(src, lab, None, cl, tr)
            assert rc == 0
            out[r64] = (lab.copy(), cl[:ncl].copy(), tr[:ntr].copy())
        finally:
            ctx.close()
    assert np.array_equal(out[True][0], out[False][0])
    _same(out[True][1], out[False][1])
    assert np.array_equal(out[True][2], out[False][2])


def test_batch_rejects_records64():
    pk = synth.generate(synth.small(shot_begin=0, n_shots=50))[0]
    ctx = tpx.Context(tpx.Config(records64=True), max_packets=pk.size)
    try:
        out = ctx.alloc_batch_outputs(pk.size, 1)
        with pytest.raises(tpx.TpxError):
            ctx.tpx_process_batch(to_device(pk), np.array([0, pk.size], np.int64), out)
    finally:
        ctx.close()
