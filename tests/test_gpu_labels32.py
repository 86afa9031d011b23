"""int32 labels (TPX_FLAG_LABELS32): the same labels as the int64 output,
minus the call's packet index base, on every path that writes them -- the
fused kernel, the general-path redo of tpx_sync, the pipelined and the
host-direct host calls -- and rejected where labels stay int64 (batches).
The allocation-free entry point's int32 labels are tested with its other
tests."""
import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import assert_clusters_equal, oracle_run, to_device

pytestmark = pytest.mark.gpu


def _labels32(ref_labels, base):
    return np.where(ref_labels < 0, -1, ref_labels - base).astype(np.int32)


@pytest.mark.parametrize("base", [0, 123_456_789_012])
def test_device_call_labels32_equal_the_oracle(base):
    pk = synth.generate(synth.small(shot_begin=0, n_shots=600, pair_frac=0.05, dark_per_shot=2.0))[0]
    ref = oracle_run(pk, index_base=base)
    ctx = tpx.Context(tpx.Config(labels32=True), max_packets=pk.size)
    try:
        r = ctx.process(to_device(pk), labels=True, is_peak=True, index_base=base, check=False)
    finally:
        ctx.close()
    assert r["status"] == 0
    assert r["labels"].dtype == np.int32
    assert np.array_equal(r["labels"], _labels32(ref["labels"], base))
    assert_clusters_equal(r["clusters"], ref["clusters"])


def test_redo_writes_labels32():
    # ToF over the whole trigger period: the fused tiles cannot hold these
    # shots, tpx_sync redoes the call on the general path
    p = synth.streaming(10e6, n_shots=40)
    pk = synth.generate(p)[0]
    base = 77
    ref = oracle_run(pk, tof_max=synth.STREAM_TOF_MAX_TICKS, index_base=base)
    ctx = tpx.Context(tpx.Config(tof_max_ticks=synth.STREAM_TOF_MAX_TICKS, labels32=True), max_packets=pk.size)
    try:
        r = ctx.process(to_device(pk), labels=True, is_peak=True, index_base=base, cluster_capacity=pk.size,
                        trig_capacity=pk.size, check=False)
    finally:
        ctx.close()
    assert r["status"] == 0 and r["counters"]["redone"] == 1
    assert np.array_equal(r["labels"], _labels32(ref["labels"], base))
    assert_clusters_equal(r["clusters"], ref["clusters"])


@pytest.mark.parametrize("direct", [False, True])
def test_host_call_labels32_equal_int64_labels(direct):
    # 2^24+ packets: the pipelined host call (pieces), or the host-direct one
    import torch
    pk = synth.generate(synth.large(n_shots=14_000))[0]
    assert pk.size >= 1 << 24
    base = 5_000_000_000
    out = {}
    for l32 in (False, True):
        ctx = tpx.Context(tpx.Config(labels32=l32, host_direct=direct), max_packets=pk.size)
        try:
            if direct:
                hp = torch.from_numpy(pk.view(np.int64)).pin_memory()
                lab_t = torch.empty(pk.size, dtype=torch.int32 if l32 else torch.int64, pin_memory=True)
                cl_t = torch.empty(pk.size // 8 * tpx.CLUSTER_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
                tr_t = torch.empty(pk.size // 8, dtype=torch.int64, pin_memory=True)
                src, lab = hp.numpy().view(np.uint64), lab_t.numpy()
                cl, tr = cl_t.numpy().view(tpx.CLUSTER_DTYPE), tr_t.numpy()
            else:
                src = pk
                lab = np.empty(pk.size, np.int32 if l32 else np.int64)
                cl = np.empty(pk.size // 8, tpx.CLUSTER_DTYPE)
                tr = np.empty(pk.size // 8, np.int64)
            rc, ncl, ntr = ctx.tpx_process_host(src, lab, None, cl, tr, index_base=base)
            assert rc == 0
            out[l32] = (lab.copy(), cl[:ncl].copy(), tr[:ntr].copy())
        finally:
            ctx.close()
    lab64, cl64, tr64 = out[False]
    lab32, cl32, tr32 = out[True]
    assert lab32.dtype == np.int32
    assert np.array_equal(lab32, _labels32(lab64, base))
    assert_clusters_equal(cl32, cl64)
    assert np.array_equal(tr32, tr64)


def test_batch_rejects_labels32():
    import torch
    pk = synth.generate(synth.small(shot_begin=0, n_shots=50))[0]
    ctx = tpx.Context(tpx.Config(labels32=True), max_packets=pk.size)
    try:
        out = ctx.alloc_batch_outputs(pk.size, 1, labels=True)
        with pytest.raises(tpx.TpxError):
            ctx.tpx_process_batch(to_device(pk), np.array([0, pk.size], np.int64), out)
    finally:
        ctx.close()
