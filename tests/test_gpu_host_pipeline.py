"""tpx_process_host on inputs large enough to be pipelined (pieces cut at
trigger packets, copies overlapping the fused kernel): the same labels,
peaks, records, triggers and counters as one device call, also when a cut
is not exact (pixels of a shot read out after the next trigger send the call
back to the one-piece path) and when the caller's record buffer is short."""
import numpy as np
import pytest

import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import COUNTERS, assert_clusters_equal, oracle_run, to_device

pytestmark = pytest.mark.gpu


def _device_call(cfg, pk):
    ctx = tpx.Context(cfg, max_packets=pk.size)
    try:
        return ctx.process(to_device(pk), labels=True, is_peak=True, cluster_capacity=pk.size // 8,
                           trig_capacity=pk.size // 8, check=False)
    finally:
        ctx.close()


def _host_call(cfg, pk, cl_cap=None, repeat=1):
    ctx = tpx.Context(cfg, max_packets=pk.size)
    try:
        lab = np.empty(pk.size, np.int64)
        peak = np.empty(pk.size, np.uint8)
        cl = np.empty(pk.size // 8 if cl_cap is None else cl_cap, tpx.CLUSTER_DTYPE)
        tr = np.empty(pk.size // 8, np.int64)
        for _ in range(repeat):
            rc, ncl, ntr = ctx.tpx_process_host(pk, lab, peak, cl, tr)
        _, counters = ctx.tpx_sync(check=False)
        return rc, ncl, ntr, lab, peak, cl, tr, counters
    finally:
        ctx.close()


def _compare(g, h):
    rc, ncl, ntr, lab, peak, cl, tr, counters = h
    assert rc == g["status"] == 0
    assert ncl == g["n_clusters"] and ntr == g["n_trig"]
    assert np.array_equal(lab, g["labels"])
    assert np.array_equal(peak, g["is_peak"])
    assert_clusters_equal(cl[:ncl], g["clusters"])
    assert np.array_equal(tr[:ntr], g["triggers"])
    for k in COUNTERS:
        assert counters[k] == g["counters"][k], k


@pytest.fixture(scope="module")
def large_stream():
    # 40,000 shots x Poisson(50): 5.1e7 packets, six pieces, pixel wraps inside
    return synth.generate(synth.large(n_shots=40_000))[0]


def test_pipelined_host_call_equals_one_device_call(large_stream):
    pk = large_stream
    cfg = tpx.Config()
    # twice on one context: the autotuner's samples, then the tuned geometry
    _compare(_device_call(cfg, pk), _host_call(cfg, pk, repeat=2))


def test_inexact_cut_falls_back_to_one_piece():
    # ToF over the whole trigger period: pixels of a shot arrive after the
    # next trigger packet, so no cut is exact (and the fused tiles cannot hold
    # these shots either: both calls end on the general path)
    p = synth.streaming(10e6, n_shots=1800)
    pk = synth.generate(p)[0]
    assert pk.size >= 1 << 24
    cfg = tpx.Config(tof_max_ticks=synth.STREAM_TOF_MAX_TICKS)
    g = _device_call(cfg, pk)
    assert g["counters"]["redone"] == 1
    _compare(g, _host_call(cfg, pk))


def test_pipelined_host_call_with_a_short_record_buffer(large_stream):
    pk = large_stream
    cfg = tpx.Config()
    g = _device_call(cfg, pk)
    cap = g["n_clusters"] // 2
    rc, ncl, ntr, lab, _, cl, tr, _ = _host_call(cfg, pk, cl_cap=cap)
    assert rc == tpx.EOVERFLOW and ncl == g["n_clusters"]
    assert_clusters_equal(cl[:cap], g["clusters"][:cap])
    assert np.array_equal(lab, g["labels"])


def test_host_direct_mode_equals_the_device_call():
    """TPX_FLAG_HOST_DIRECT: with every host buffer pinned (mapped into the
    device), the fused kernel works on them in place; the result equals the
    oracle's. A pageable buffer makes the call stage through the device as
    usual, with the same result."""
    import torch
    pk = synth.generate(synth.large(n_shots=600))[0]
    o = oracle_run(pk)
    n = pk.size
    h_pk = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_pk.numpy()[:] = pk.view(np.int64)
    lab = torch.empty(n, dtype=torch.int64, pin_memory=True)
    cl = torch.empty(n // 8 * tpx.CLUSTER_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    tr = torch.empty(1000, dtype=torch.int64, pin_memory=True)
    ctx = tpx.Context(tpx.Config(host_direct=True), max_packets=n)
    try:
        for labels in (lab.numpy(), np.empty(n, np.int64)):       # pinned, then pageable labels
            a_cl = cl.numpy().view(tpx.CLUSTER_DTYPE)
            rc, ncl, ntr = ctx.tpx_process_host(h_pk.numpy().view(np.uint64), labels, None, a_cl, tr.numpy())
            assert rc == 0
            assert np.array_equal(labels, o["labels"])
            assert np.array_equal(tr.numpy()[:ntr], o["triggers"])
            assert ncl == o["clusters"].size
            assert_clusters_equal(a_cl[:ncl].copy(), o["clusters"])
    finally:
        ctx.close()
