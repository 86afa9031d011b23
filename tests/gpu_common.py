"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI and compare it with the oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2603_04942_gb300 as tpx

INT_FIELDS = ("label", "shot", "t0", "s_tot", "s_x", "s_y", "s_t", "n", "n_peaks")
FLOAT_FIELDS = ("x", "y", "tof")
# Integer sums are exact; the final double division of Sec. V.C is allowed
# 1e-6 px (and 1e-6 tick) -- both sides compute s/S_tot with one IEEE division.
TOL = 1e-6


def to_device(pk: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pk).view(np.int64)).cuda()


def gpu_run(pk: np.ndarray, *, rx=1, ry=1, dt=32, mode=0, tof_max=64_000, lut=None, strict=False,
            index_base=0, labels=True, is_peak=True, cluster_capacity=None, trig_capacity=None, tile=0):
    import torch
    dlut = None if lut is None else torch.from_numpy(np.asarray(lut, np.int16)).cuda()
    cfg = tpx.Config(rx=rx, ry=ry, dt_ticks=dt, mode=mode, tof_max_ticks=tof_max, timewalk_lut=dlut,
                     strict=strict, tile_geometry=tile)
    ctx = tpx.Context(cfg, max_packets=max(1, pk.size))
    try:
        d = to_device(pk) if pk.size else torch.zeros(2, dtype=torch.int64, device="cuda")
        out = ctx.alloc_outputs(pk.size, labels, is_peak,
                                cluster_capacity if cluster_capacity is not None else max(16, pk.size),
                                trig_capacity if trig_capacity is not None else max(16, pk.size))
        ctx.tpx_process(d, out, index_base, n_packets=pk.size)
        rc, counters = ctx.tpx_sync(check=False)
        return ctx.collect(out, rc, counters)
    finally:
        ctx.close()


def oracle_run(pk, *, rx=1, ry=1, dt=32, mode=0, tof_max=64_000, lut=None, strict=False, index_base=0):
    cfg = oracle.Config(rx=rx, ry=ry, dt_ticks=dt, mode=mode, tof_max_ticks=tof_max, timewalk_lut=lut,
                        strict=strict)
    return oracle.run(pk, cfg, idx_base=index_base)


def assert_clusters_equal(gc: np.ndarray, oc: np.ndarray):
    assert gc.size == oc.size, (gc.size, oc.size)
    for f in INT_FIELDS:
        if not np.array_equal(gc[f], oc[f]):
            bad = np.flatnonzero(gc[f] != oc[f])[:5]
            raise AssertionError(f"field {f} differs at {bad}: gpu {gc[bad]} oracle {oc[bad]}")
    for f in FLOAT_FIELDS:
        g, o = gc[f], oc[f]
        same_nan = np.isnan(g) & np.isnan(o)
        ok = same_nan | (np.abs(g - o) <= TOL)
        assert ok.all(), (f, np.flatnonzero(~ok)[:5])


COUNTERS = ("pixels", "tdcs", "corrupt", "dropped_pre_trigger", "dropped_background", "kept", "clusters",
            "peaks")  # "redone" and "status_bits" describe the path, not the result


def assert_parity(g: dict, o: dict, check_counters=True):
    assert np.array_equal(g["triggers"], o["triggers"])
    assert g["n_trig"] == o["triggers"].size
    assert np.array_equal(g["labels"], o["labels"]), np.flatnonzero(g["labels"] != o["labels"])[:10]
    if g["is_peak"] is not None:
        assert np.array_equal(g["is_peak"], o["is_peak"]), np.flatnonzero(g["is_peak"] != o["is_peak"])[:10]
    assert g["n_clusters"] == o["clusters"].size
    assert_clusters_equal(g["clusters"], o["clusters"])
    if check_counters:
        for k in COUNTERS:
            assert g["counters"][k] == o["counters"][k], (k, g["counters"][k], o["counters"][k])
