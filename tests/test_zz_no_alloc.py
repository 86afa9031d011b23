"""tpx_process_noalloc: the fused path for callers that cannot allocate
device memory where they process data -- acquisition loops that must not
block in the allocator, or hosts that fix the library's memory budget up
front. Its look-back scratch is one fixed array in the library image.

Called through the C ABI, its output must equal the oracle's and tpx_process's
on the same input on two calls in a row (the shared fixed scratch keeps the
previous call's contents, which must not leak into the next result), also
when the calls cross the wrap of the look-back sequence number. A shot longer
than a tile's range returns TPX_EUNSUPPORTED (no redo). Collected last so that
a stop-at-first-failure run has already run every other test; it passes alone
in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_common import TOL, INT_FIELDS, FLOAT_FIELDS, assert_clusters_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

NOALLOC_MAX_PACKETS = 1 << 26


def _lib():
    import paper_2603_04942_gb300 as tpx
    from paper_2603_04942_gb300 import build as b
    b.build()
    L = tpx.load()
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.tpx_process_noalloc.argtypes = [ctypes.POINTER(tpx._CConfig), vp, vp, i64, i64, vp, vp, vp, i64, vp, vp,
                                      i64, vp, ctypes.POINTER(tpx._CCounters)]
    L.tpx_process_noalloc.restype = ctypes.c_int
    L.tpx_debug_noalloc_seq.argtypes = [ctypes.c_uint32]
    L.tpx_debug_noalloc_seq.restype = ctypes.c_int
    return tpx, L


def _noalloc_run(tpx, L, pk, cfg, index_base=0):
    import torch
    n = pk.size
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    cl_cap, tr_cap = max(16, n), max(16, n)
    labels = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    is_peak = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    clusters = torch.zeros(cl_cap * tpx.CLUSTER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    trig = torch.zeros(tr_cap, dtype=torch.int64, device="cuda")
    n_cl = torch.zeros(1, dtype=torch.int64, device="cuda")
    n_tr = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = tpx._CCounters()
    torch.cuda.synchronize()
    rc = L.tpx_process_noalloc(ctypes.byref(cfg), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               d.data_ptr(), n, index_base, labels.data_ptr(), is_peak.data_ptr(),
                               clusters.data_ptr(), cl_cap, n_cl.data_ptr(), trig.data_ptr(), tr_cap,
                               n_tr.data_ptr(), ctypes.byref(cnt))
    ncl, ntr = int(n_cl.item()), int(n_tr.item())
    raw = clusters[: min(ncl, cl_cap) * tpx.CLUSTER_DTYPE.itemsize].cpu().numpy()
    return dict(status=rc, labels=labels.cpu().numpy(), is_peak=is_peak.cpu().numpy(),
                clusters=np.frombuffer(raw.tobytes(), tpx.CLUSTER_DTYPE).copy(), n_clusters=ncl,
                triggers=trig[:ntr].cpu().numpy(), counters={f: int(getattr(cnt, f)) for f in
                                                             ("kept", "clusters", "peaks", "pixels")})


def _same(a, b):
    """Two GPU results (this call and tpx_process) agree element by element."""
    assert a["status"] == 0 and b["status"] == 0
    assert np.array_equal(a["labels"], b["labels"])
    assert np.array_equal(a["is_peak"], b["is_peak"])
    assert np.array_equal(a["triggers"], b["triggers"])
    assert a["n_clusters"] == b["n_clusters"] == a["clusters"].size == b["clusters"].size
    for f in INT_FIELDS:
        assert np.array_equal(a["clusters"][f], b["clusters"][f]), f
    for f in FLOAT_FIELDS:
        assert np.all(np.abs(a["clusters"][f] - b["clusters"][f]) <= TOL), f


def _matches_oracle(g, o):
    """This call against the CPU oracle: labels, peaks, triggers bit-exact;
    records' integer fields bit-exact, centroids within 1e-6."""
    assert g["status"] == 0 and o["status"] == 0
    assert np.array_equal(g["labels"], o["labels"])
    assert np.array_equal(g["is_peak"], o["is_peak"])
    assert np.array_equal(g["triggers"], o["triggers"])
    assert g["n_clusters"] == o["clusters"].size
    assert_clusters_equal(g["clusters"], o["clusters"])
    assert g["counters"]["kept"] == o["counters"]["kept"]
    assert g["counters"]["peaks"] == o["counters"]["peaks"]


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_oracle_and_tpx_process_twice(mode):
    tpx, L = _lib()
    pk = synth.generate(synth.large(n_shots=300, dark_per_shot=2.0))[0]
    o = oracle_run(pk, mode=mode, index_base=5)
    ref = gpu_run(pk, mode=mode, index_base=5)
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    cfg.mode = mode
    first = _noalloc_run(tpx, L, pk, cfg, index_base=5)
    second = _noalloc_run(tpx, L, pk, cfg, index_base=5)
    _matches_oracle(first, o)
    _matches_oracle(second, o)
    _same(first, ref)
    _same(second, ref)
    # a different, smaller input right after: nothing of the previous call leaks
    pk2 = pk[: 3 * 4096 + 11]
    _matches_oracle(_noalloc_run(tpx, L, pk2, cfg), oracle_run(pk2, mode=mode))


def test_noalloc_calls_across_the_sequence_wrap():
    """The look-back flags carry a 30-bit call sequence number; where it wraps
    the fixed array's flags are cleared. Calls just before, at and after the
    wrap all equal the oracle."""
    tpx, L = _lib()
    pk = synth.generate(synth.large(n_shots=200, seed=11))[0]
    o = oracle_run(pk)
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    assert L.tpx_debug_noalloc_seq((1 << 30) - 2) == 0
    for _ in range(3):     # sequence numbers 2^30 - 1, then 1 (after the clear), then 2
        _matches_oracle(_noalloc_run(tpx, L, pk, cfg), o)
    assert L.tpx_debug_noalloc_seq(1 << 30) == tpx.EINVAL


def test_noalloc_shot_beyond_a_range_is_unsupported():
    """A shot of more than 8192 packets does not fit a tile's range; tpx_sync
    would redo such a call with the general path, this call returns
    TPX_EUNSUPPORTED. The next ordinary call is exact again."""
    tpx, L = _lib()
    long_pk = synth.generate(synth.small(n_shots=3, particles_per_shot=600.0, seed=12))[0]
    tdc = np.flatnonzero((long_pk >> np.uint64(60)) == 6)
    assert np.diff(np.r_[tdc, long_pk.size]).max() > 8192
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    assert _noalloc_run(tpx, L, long_pk, cfg)["status"] == tpx.EUNSUPPORTED
    pk = synth.generate(synth.small(n_shots=50, seed=13))[0]
    _matches_oracle(_noalloc_run(tpx, L, pk, cfg), oracle_run(pk))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    tpx, L = _lib()
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    dummy = ctypes.c_int64()
    rc = L.tpx_process_noalloc(ctypes.byref(cfg), None, None, NOALLOC_MAX_PACKETS + 1, 0, None, None, None, 0,
                               ctypes.addressof(dummy), None, 0, ctypes.addressof(dummy), None)
    assert rc == tpx.EINVAL


def test_labels32_equal_the_oracle():
    import torch
    tpx, L = _lib()
    pk = synth.generate(synth.small(shot_begin=0, n_shots=300))[0]
    base = 1000
    ref = oracle_run(pk, index_base=base)
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    cfg.flags = tpx.FLAG_LABELS32
    n = pk.size
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    labels = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    clusters = torch.zeros(n * tpx.CLUSTER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    trig = torch.zeros(n, dtype=torch.int64, device="cuda")
    n_cl = torch.zeros(1, dtype=torch.int64, device="cuda")
    n_tr = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = tpx._CCounters()
    torch.cuda.synchronize()
    rc = L.tpx_process_noalloc(ctypes.byref(cfg), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               d.data_ptr(), n, base, labels.data_ptr(), None, clusters.data_ptr(), n,
                               n_cl.data_ptr(), trig.data_ptr(), n, n_tr.data_ptr(), ctypes.byref(cnt))
    assert rc == 0
    want = np.where(ref["labels"] < 0, -1, ref["labels"] - base).astype(np.int32)
    assert np.array_equal(labels.cpu().numpy(), want)
    ncl = int(n_cl.item())
    g = np.frombuffer(clusters[: ncl * tpx.CLUSTER_DTYPE.itemsize].cpu().numpy().tobytes(), tpx.CLUSTER_DTYPE)
    assert_clusters_equal(g, ref["clusters"])


def test_records64_equal_the_oracle():
    import torch
    tpx, L = _lib()
    pk = synth.generate(synth.small(shot_begin=0, n_shots=300))[0]
    ref = oracle_run(pk)
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    cfg.flags = tpx.FLAG_RECORDS64
    n = pk.size
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    labels = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    clusters = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    trig = torch.zeros(n, dtype=torch.int64, device="cuda")
    n_cl = torch.zeros(1, dtype=torch.int64, device="cuda")
    n_tr = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = tpx._CCounters()
    torch.cuda.synchronize()
    rc = L.tpx_process_noalloc(ctypes.byref(cfg), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               d.data_ptr(), n, 0, labels.data_ptr(), None, clusters.data_ptr(), n,
                               n_cl.data_ptr(), trig.data_ptr(), n, n_tr.data_ptr(), ctypes.byref(cnt))
    assert rc == 0
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    ncl = int(n_cl.item())
    g = np.frombuffer(clusters[: ncl * 64].cpu().numpy().tobytes(), tpx.CLUSTER64_DTYPE)
    assert g.size == ref["clusters"].size
    for f in tpx.CLUSTER64_DTYPE.names:
        assert np.array_equal(g[f], ref["clusters"][f]), f
