"""Python binding of libtpx, the GB300 TPX3 clustering / centroiding library.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch provides device memory and the CUDA stream. The entry points
have the C-ABI names of include/tpx.h (tpx_create, tpx_process,
tpx_process_host, tpx_sync, ...). There is no CPU fallback: if the library or
a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build_mod

__all__ = ["Config", "Context", "CLUSTER_DTYPE", "TpxError", "lib", "load", "MODE_CC", "MODE_PAPER",
           "EXPORTED_SYMBOLS"]

MODE_CC = 0
MODE_PAPER = 1
TILE_DEFAULT, TILE_4096, TILE_2048 = 0, 1, 2
FLAG_HOST_DIRECT = 4
FLAG_LABELS32 = 8
FLAG_RECORDS64 = 16
TICK_NS = 1.5625

OK, EINVAL, ENOMEM, EOVERFLOW, ECORRUPT, EAGAIN, ETIMEOUT, EDEVTIMEOUT, ECUDA, EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9

# tpx_record, 88 bytes, ascending label order
CLUSTER_DTYPE = np.dtype([("label", "<i8"), ("shot", "<i8"), ("t0", "<i8"), ("s_tot", "<i8"),
                          ("s_x", "<i8"), ("s_y", "<i8"), ("s_t", "<i8"), ("n", "<i4"),
                          ("n_peaks", "<i4"), ("x", "<f8"), ("y", "<f8"), ("tof", "<f8")])
assert CLUSTER_DTYPE.itemsize == 88
# tpx_record64 (TPX_FLAG_RECORDS64): the record without the derived x, y, tof
CLUSTER64_DTYPE = np.dtype([("label", "<i8"), ("shot", "<i8"), ("t0", "<i8"), ("s_tot", "<i8"),
                            ("s_x", "<i8"), ("s_y", "<i8"), ("s_t", "<i8"), ("n", "<i4"), ("n_peaks", "<i4")])
assert CLUSTER64_DTYPE.itemsize == 64

COUNTER_FIELDS = ("packets", "pixels", "tdcs", "corrupt", "dropped_pre_trigger", "dropped_background",
                  "kept", "clusters", "peaks", "status_bits", "redone")

EXPORTED_SYMBOLS = ("tpx_config_default", "tpx_create", "tpx_reserve", "tpx_destroy", "tpx_process",
                    "tpx_process_host", "tpx_sync", "tpx_kernel_timing", "tpx_kernel_times", "tpx_debug_phase_times", "tpx_process_noalloc", "tpx_decode", "tpx_cluster",
                    "tpx_centroid", "tpx_tuning", "tpx_process_batch", "tpx_tot_tof_histogram", "tpx_refine_patches", "tpx_refiner_params",
                    "tpx_refiner_forward", "tpx_refiner_train_step", "tpx_refine_decide",
                    "tpx_refiner_packed_bytes", "tpx_refiner_pack", "tpx_refiner_infer", "tpx_debug_hold_tile", "tpx_debug_noalloc_seq", "tpx_set_state", "tpx_get_state", "tpx_summarize", "tpx_stream_create",
                    "tpx_stream_submit", "tpx_stream_finish", "tpx_stream_poll", "tpx_stream_destroy",
                    "tpx_stream_snapshot_bytes", "tpx_stream_snapshot", "tpx_stream_restore",
                    "tpx_cnn_params", "tpx_cnn_work_floats", "tpx_cnn_forward", "tpx_cnn_train_step",
                    "tpx_cnn_packed_bytes", "tpx_cnn_pack", "tpx_cnn_infer_work_bytes", "tpx_cnn_infer", "tpx_debug_cnn_phase_times",
                    "tpx_refine_patches_bf16", "tpx_strerror", "tpx_version")


class _CConfig(ctypes.Structure):
    _fields_ = [("rx", ctypes.c_int32), ("ry", ctypes.c_int32), ("dt_ticks", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("tof_max_ticks", ctypes.c_int64),
                ("wrap_thr_pix_ticks", ctypes.c_int64), ("wrap_thr_tdc_ticks", ctypes.c_int64),
                ("d_timewalk_lut", ctypes.c_void_p), ("strict", ctypes.c_int32), ("chain", ctypes.c_int32),
                ("tile_geometry", ctypes.c_int32), ("flags", ctypes.c_int32)]


STATE_FIELDS = ("pixels", "pix_last_raw", "pix_wraps", "triggers", "tdc_last_raw", "tdc_wraps")


class _CState(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in STATE_FIELDS]


SUMMARY_FIELDS = ("pixels", "pix_first_raw", "pix_last_raw", "pix_wraps",
                  "triggers", "tdc_first_raw", "tdc_last_raw", "tdc_wraps")


class _CSummary(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in SUMMARY_FIELDS]


class _CCounters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in COUNTER_FIELDS]


class _CHits(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("index", "shot", "t", "tof", "x", "y", "tot")]


class _CStreamConfig(ctypes.Structure):
    _fields_ = [("cfg", _CConfig), ("max_chunk_packets", ctypes.c_int64), ("max_hold_packets", ctypes.c_int64),
                ("hold_triggers", ctypes.c_int32), ("slots", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64)]


class _CStreamResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("first_shot", ctypes.c_int64), ("n_shots", ctypes.c_int64), ("trig_t", ctypes.c_void_p),
                ("n_clusters", ctypes.c_int64), ("clusters", ctypes.c_void_p),
                ("packets_processed", ctypes.c_int64), ("latency_us", ctypes.c_double)]


class TpxError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {lib().tpx_strerror(code).decode()} ({code})")


@dataclasses.dataclass
class Config:
    """Mirror of tpx_config (Sec. IV.A-C and V.A parameters)."""
    rx: int = 1
    ry: int = 1
    dt_ticks: int = 32
    mode: int = MODE_CC
    tof_max_ticks: int = 64_000
    wrap_thr_pix_ticks: int = 12_800_000_000
    wrap_thr_tdc_ticks: int = 12_800_000_000
    timewalk_lut: object = None        # torch int16 tensor of 1024 on the device, or None
    strict: bool = False
    chain: bool = False                # each call continues where the previous one ended
    tile_geometry: int = 0             # TILE_DEFAULT, TILE_4096 or TILE_2048 (speed only)
    host_direct: bool = False          # tpx_process_host on mapped pinned host buffers in place
    labels32: bool = False             # per-packet labels as int32, relative to the call's index base
    records64: bool = False            # 64-byte records (CLUSTER64_DTYPE: no x, y, tof)

    def flags(self) -> int:
        return ((FLAG_HOST_DIRECT if self.host_direct else 0) | (FLAG_LABELS32 if self.labels32 else 0) |
                (FLAG_RECORDS64 if self.records64 else 0))

    def record_dtype(self) -> np.dtype:
        return CLUSTER64_DTYPE if self.records64 else CLUSTER_DTYPE


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the built library; raise if it is missing (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build_mod.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libtpx is not built ({path}); run paper_2603_04942_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.tpx_config_default.argtypes = [ctypes.POINTER(_CConfig)]
        L.tpx_config_default.restype = None
        L.tpx_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_CConfig), i64, vp]
        L.tpx_reserve.argtypes = [vp, i64]
        L.tpx_destroy.argtypes = [vp]
        L.tpx_process.argtypes = [vp, vp, i64, i64, vp, vp, vp, i64, vp, vp, i64, vp]
        L.tpx_process_host.argtypes = [vp, vp, i64, i64, vp, vp, vp, i64, vp, vp, i64, vp]
        L.tpx_sync.argtypes = [vp, ctypes.POINTER(_CCounters)]
        L.tpx_kernel_timing.argtypes = [vp, i32]
        L.tpx_debug_phase_times.argtypes = [i32, ctypes.POINTER(ctypes.c_uint64), i32]
        L.tpx_debug_phase_times.restype = i32
        L.tpx_debug_cnn_phase_times.argtypes = [ctypes.POINTER(ctypes.c_uint64), i32]
        L.tpx_debug_cnn_phase_times.restype = i32
        L.tpx_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]
        L.tpx_strerror.argtypes = [i32]
        L.tpx_strerror.restype = ctypes.c_char_p
        L.tpx_version.restype = ctypes.c_char_p
        L.tpx_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.tpx_process_batch.argtypes = [vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp]
        L.tpx_tot_tof_histogram.argtypes = [vp, ctypes.POINTER(_CHits), i64, i32, i32, i32, vp]
        L.tpx_refine_patches.argtypes = [vp, vp, i64, i64, vp, vp, i64, i32, vp, vp, vp, i64, vp]
        L.tpx_refiner_params.argtypes = [i32]
        L.tpx_refiner_params.restype = i64
        L.tpx_refiner_forward.argtypes = [vp, vp, i32, vp, i64, vp, vp]
        L.tpx_refiner_train_step.argtypes = [vp, vp, vp, vp, vp, i32, i64, vp, vp, i64, ctypes.c_float,
                                             ctypes.c_float, vp, vp]
        L.tpx_refine_decide.argtypes = [vp, vp, vp, vp, vp, i64, ctypes.c_float, vp]
        L.tpx_debug_hold_tile.argtypes = [vp, i64]
        L.tpx_debug_hold_tile.restype = i32
        L.tpx_refiner_packed_bytes.argtypes = [i32]
        L.tpx_refiner_packed_bytes.restype = i64
        L.tpx_refiner_pack.argtypes = [vp, vp, i32, vp]
        L.tpx_refiner_infer.argtypes = [vp, vp, i32, vp, i64, vp]
        for f in ("tpx_refine_patches", "tpx_refiner_forward", "tpx_refiner_train_step", "tpx_refine_decide",
                  "tpx_refiner_pack", "tpx_refiner_infer"):
            getattr(L, f).restype = i32
        L.tpx_refine_patches_bf16.argtypes = [vp, vp, i64, i64, vp, vp, i64, i32, vp, vp, vp, i64, vp]
        L.tpx_refine_patches_bf16.restype = i32
        for f in ("tpx_cnn_params", "tpx_cnn_packed_bytes"):
            getattr(L, f).argtypes = []
            getattr(L, f).restype = i64
        for f in ("tpx_cnn_work_floats", "tpx_cnn_infer_work_bytes"):
            getattr(L, f).argtypes = [i64]
            getattr(L, f).restype = i64
        L.tpx_cnn_forward.argtypes = [vp, vp, vp, i64, vp, vp]
        L.tpx_cnn_train_step.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, i64, ctypes.c_float, ctypes.c_float, vp, vp]
        L.tpx_cnn_pack.argtypes = [vp, vp, vp]
        L.tpx_cnn_infer.argtypes = [vp, vp, vp, i64, vp, vp]
        for f in ("tpx_cnn_forward", "tpx_cnn_train_step", "tpx_cnn_pack", "tpx_cnn_infer"):
            getattr(L, f).restype = i32
        L.tpx_set_state.argtypes = [vp, ctypes.POINTER(_CState)]
        L.tpx_get_state.argtypes = [vp, ctypes.POINTER(_CState)]
        L.tpx_set_state.restype = i32
        L.tpx_get_state.restype = i32
        L.tpx_summarize.argtypes = [vp, vp, i64, ctypes.POINTER(_CSummary)]
        L.tpx_summarize.restype = i32
        L.tpx_stream_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_CStreamConfig), vp]
        L.tpx_stream_submit.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
        L.tpx_stream_finish.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.tpx_stream_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_CStreamResult), ctypes.c_int32]
        L.tpx_stream_destroy.argtypes = [vp]
        L.tpx_stream_snapshot_bytes.argtypes = [vp]
        L.tpx_stream_snapshot_bytes.restype = i64
        L.tpx_stream_snapshot.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.tpx_stream_snapshot.restype = i32
        L.tpx_stream_restore.argtypes = [vp, vp, i64]
        L.tpx_stream_restore.restype = i32
        for f in ("tpx_stream_create", "tpx_stream_submit", "tpx_stream_finish", "tpx_stream_poll",
                  "tpx_stream_destroy"):
            getattr(L, f).restype = i32
        L.tpx_decode.argtypes = [vp, vp, i64, i64, ctypes.POINTER(_CHits), i64, vp, vp, i64, vp]
        L.tpx_cluster.argtypes = [vp, ctypes.POINTER(_CHits), i64, vp, vp]
        L.tpx_centroid.argtypes = [vp, ctypes.POINTER(_CHits), vp, vp, i64, vp, i64, vp]
        for f in ("tpx_create", "tpx_reserve", "tpx_destroy", "tpx_process", "tpx_process_host", "tpx_sync",
                  "tpx_kernel_timing", "tpx_kernel_times", "tpx_decode", "tpx_cluster", "tpx_centroid"):
            getattr(L, f).restype = i32
        _lib = L
        return L


def lib():
    return load()


PHASE_NAMES = ("tile start", "tile load", "look-ahead", "walk 2 and its scan", "trigger times",
               "walk 4 (records)", "hash insert", "neighbour pass", "compression", "unions", "roots",
               "member lists", "member-list walks (and the previous tile's copy-out)",
               "staged stores", "labels and offsets", "tail", "CTA end",
               "big ranges (batches: the sorted-window path)", "big ranges: the previous tile's copy-out",
               "label ranks (bitmap scan)", "big: range end, walk 2, triggers", "big: walk 4", "big: bins and sort",
               "big: neighbour pass", "big: compression and roots", "big: moments", "big: labels, records, outputs")


CNN_PHASE_NAMES = ("wait for the patches", "conversion to the conv1 map", "conv1 MMAs", "conv1 epilogue",
                   "conv2 MMAs", "conv2 epilogue", "conv3 MMAs", "conv3 epilogue", "fc1 MMAs", "fc1 epilogue",
                   "fc2 MMAs", "fc2 epilogue")


def cnn_phase_times(clear: bool = True) -> np.ndarray:
    """The CNN inference kernel's per-phase cycle counters (instrumented build only)."""
    arr = (ctypes.c_uint64 * 16)()
    rc = lib().tpx_debug_cnn_phase_times(arr, 1 if clear else 0)
    if rc:
        raise TpxError(rc, "tpx_debug_cnn_phase_times")
    return np.array(arr[:len(CNN_PHASE_NAMES)], dtype=np.uint64)


def phase_times(tile_geometry: int, clear: bool = True) -> np.ndarray:
    """The fused kernel's per-phase cycle counters (instrumented build only)."""
    arr = (ctypes.c_uint64 * 32)()
    rc = lib().tpx_debug_phase_times(int(tile_geometry), arr, 1 if clear else 0)
    if rc:
        raise TpxError(rc, "tpx_debug_phase_times")
    return np.array(arr[:len(PHASE_NAMES)], dtype=np.uint64)


def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


class Context:
    """A tpx_ctx bound to a torch CUDA stream."""

    def __init__(self, cfg: Config | None = None, max_packets: int = 1 << 20, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libtpx needs a CUDA device")
        self.cfg = cfg or Config()
        self._lut = self.cfg.timewalk_lut
        if self._lut is not None:
            assert self._lut.dtype == torch.int16 and self._lut.numel() == 1024 and self._lut.is_cuda
        c = _CConfig(self.cfg.rx, self.cfg.ry, self.cfg.dt_ticks, self.cfg.mode, self.cfg.tof_max_ticks,
                     self.cfg.wrap_thr_pix_ticks, self.cfg.wrap_thr_tdc_ticks, _ptr(self._lut),
                     int(self.cfg.strict), int(self.cfg.chain), int(self.cfg.tile_geometry),
                     self.cfg.flags())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = lib().tpx_create(ctypes.byref(h), ctypes.byref(c), int(max_packets), ctypes.c_void_p(self.stream.cuda_stream))
        if rc:
            raise TpxError(rc, "tpx_create")
        self._h = h

    def reserve(self, max_packets: int):
        rc = lib().tpx_reserve(self._h, int(max_packets))
        if rc:
            raise TpxError(rc, "tpx_reserve")

    def tpx_tuning(self) -> dict:
        """The tile geometry in use (0 while the autotuner samples) and the
        best measured ms per 10^6 packets of the 4096- and 2048-packet tiles."""
        g = ctypes.c_int32(0)
        ms = (ctypes.c_double * 2)()
        rc = lib().tpx_tuning(self._h, ctypes.byref(g), ms)
        if rc:
            raise TpxError(rc, "tpx_tuning")
        return {"tile_geometry": int(g.value), "ms_per_mpacket": {"4096": ms[0], "2048": ms[1]}}

    def tpx_set_state(self, state: dict | None):
        st = None if state is None else _CState(*(int(state[f]) for f in STATE_FIELDS))
        rc = lib().tpx_set_state(self._h, ctypes.byref(st) if st is not None else None)
        if rc:
            raise TpxError(rc, "tpx_set_state")

    def tpx_get_state(self) -> dict:
        st = _CState()
        rc = lib().tpx_get_state(self._h, ctypes.byref(st))
        if rc:
            raise TpxError(rc, "tpx_get_state")
        return {f: int(getattr(st, f)) for f in STATE_FIELDS}

    def tpx_summarize(self, packets, n_packets: int | None = None) -> dict:
        """Associative unwrap summary of a packet range (see shard.py)."""
        n = int(packets.numel() if n_packets is None else n_packets)
        out = _CSummary()
        rc = lib().tpx_summarize(self._h, _ptr(packets), n, ctypes.byref(out))
        if rc:
            raise TpxError(rc, "tpx_summarize")
        return {f: int(getattr(out, f)) for f in SUMMARY_FIELDS}

    def close(self):
        if getattr(self, "_h", None):
            lib().tpx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device buffers (asynchronous; call sync() to read the status) --
    def alloc_outputs(self, n_packets: int, labels=True, is_peak=False, cluster_capacity=None,
                      trig_capacity=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        cl_cap = int(cluster_capacity if cluster_capacity is not None else max(16, n_packets // 4))
        tr_cap = int(trig_capacity if trig_capacity is not None else max(16, n_packets // 8))
        return dict(
            labels=torch.empty(n_packets, dtype=torch.int32 if self.cfg.labels32 else torch.int64,
                               device=dev) if labels else None,
            is_peak=torch.empty(n_packets, dtype=torch.uint8, device=dev) if is_peak else None,
            clusters=torch.empty(cl_cap * self.cfg.record_dtype().itemsize, dtype=torch.uint8, device=dev),
            n_clusters=torch.zeros(1, dtype=torch.int64, device=dev),
            trig=torch.empty(tr_cap, dtype=torch.int64, device=dev),
            n_trig=torch.zeros(1, dtype=torch.int64, device=dev),
            cluster_capacity=cl_cap, trig_capacity=tr_cap, record_dtype=self.cfg.record_dtype())

    def tpx_process(self, packets, out: dict, index_base: int = 0, n_packets: int | None = None):
        n = int(packets.numel() if n_packets is None else n_packets)
        rc = lib().tpx_process(self._h, _ptr(packets), n, int(index_base), _ptr(out["labels"]),
                               _ptr(out["is_peak"]), _ptr(out["clusters"]), out["cluster_capacity"],
                               _ptr(out["n_clusters"]), _ptr(out["trig"]), out["trig_capacity"],
                               _ptr(out["n_trig"]))
        if rc:
            raise TpxError(rc, "tpx_process")

    # -- batches of independent runs, one launch --
    def alloc_batch_outputs(self, n_packets: int, n_runs: int, labels=False, is_peak=False, cluster_capacity=None,
                            trig_capacity=None) -> dict:
        import torch
        out = self.alloc_outputs(n_packets, labels, is_peak, cluster_capacity, trig_capacity)
        dev = out["n_clusters"].device
        out["run_clusters"] = torch.zeros(n_runs + 1, dtype=torch.int64, device=dev)
        out["run_trig"] = torch.zeros(n_runs + 1, dtype=torch.int64, device=dev)
        return out

    def tpx_process_batch(self, packets, run_offsets: np.ndarray, out: dict):
        """Runs [run_offsets[r], run_offsets[r+1]) of the device packets, each
        a stream of its own, in one launch (host int64 offsets)."""
        offs = np.ascontiguousarray(run_offsets, dtype=np.int64)
        self._batch_offs = offs   # the call reads them before it returns; kept for the caller's reference
        rc = lib().tpx_process_batch(self._h, _ptr(packets), offs.ctypes.data, offs.size - 1, _ptr(out["labels"]),
                                     _ptr(out["is_peak"]), _ptr(out["clusters"]), out["cluster_capacity"],
                                     _ptr(out["n_clusters"]), _ptr(out["run_clusters"]), _ptr(out["trig"]),
                                     out["trig_capacity"], _ptr(out["n_trig"]), _ptr(out["run_trig"]))
        if rc:
            raise TpxError(rc, "tpx_process_batch")

    @staticmethod
    def collect_batch(out: dict, rc: int, counters: dict) -> dict:
        r = Context.collect(out, rc, counters)
        r["run_clusters"] = out["run_clusters"].cpu().numpy()
        r["run_trig"] = out["run_trig"].cpu().numpy()
        return r

    def tpx_sync(self, check: bool = True) -> tuple[int, dict]:
        cnt = _CCounters()
        rc = lib().tpx_sync(self._h, ctypes.byref(cnt))
        counters = {f: int(getattr(cnt, f)) for f in COUNTER_FIELDS}
        if check and rc:
            raise TpxError(rc, "tpx_sync")
        return rc, counters

    def tpx_kernel_timing(self, enable: bool = True) -> None:
        rc = lib().tpx_kernel_timing(self._h, 1 if enable else 0)
        if rc:
            raise TpxError(rc, "tpx_kernel_timing")

    def tpx_kernel_times(self) -> dict:
        """Summed CUDA-event times of the fused launches since timing was
        enabled: {"prepass_ms", "fused_ms", "launches"}."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        rc = lib().tpx_kernel_times(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n))
        if rc:
            raise TpxError(rc, "tpx_kernel_times")
        return {"prepass_ms": a.value, "fused_ms": b.value, "launches": n.value}

    def process(self, packets, labels=True, is_peak=False, cluster_capacity=None, trig_capacity=None,
                index_base: int = 0, check: bool = True) -> dict:
        """Run the fused path on device-resident packets and return host
        copies: clusters (structured numpy array), labels, is_peak,
        triggers, counters and the status code."""
        n = int(packets.numel())
        if n > self.max_packets_hint():
            self.reserve(n)
        out = self.alloc_outputs(n, labels, is_peak, cluster_capacity, trig_capacity)
        self.tpx_process(packets, out, index_base)
        rc, counters = self.tpx_sync(check=check)
        return self.collect(out, rc, counters)

    def max_packets_hint(self) -> int:
        return 1 << 62

    @staticmethod
    def collect(out: dict, rc: int, counters: dict) -> dict:
        ncl = int(out["n_clusters"].item())
        ntr = int(out["n_trig"].item())
        m = min(ncl, out["cluster_capacity"])
        dt = out.get("record_dtype", CLUSTER_DTYPE)
        raw = out["clusters"][: m * dt.itemsize].cpu().numpy()
        clusters = np.frombuffer(raw.tobytes(), dt).copy() if m else np.zeros(0, dt)
        return dict(status=rc, counters=counters, clusters=clusters, n_clusters=ncl, n_trig=ntr,
                    triggers=out["trig"][: min(ntr, out["trig_capacity"])].cpu().numpy(),
                    labels=None if out["labels"] is None else out["labels"].cpu().numpy(),
                    is_peak=None if out["is_peak"] is None else out["is_peak"].cpu().numpy())

    # -- host buffers (the end-to-end call) --
    def tpx_process_host(self, packets: np.ndarray, labels: np.ndarray | None, is_peak: np.ndarray | None,
                         clusters: np.ndarray, triggers: np.ndarray, index_base: int = 0) -> tuple[int, int, int]:
        assert packets.dtype == np.uint64 and packets.flags.c_contiguous
        assert labels is None or labels.dtype == (np.int32 if self.cfg.labels32 else np.int64)
        assert clusters.dtype == self.cfg.record_dtype()
        n_cl = ctypes.c_int64()
        n_tr = ctypes.c_int64()
        rc = lib().tpx_process_host(self._h, packets.ctypes.data, packets.size, int(index_base),
                                    None if labels is None else labels.ctypes.data,
                                    None if is_peak is None else is_peak.ctypes.data,
                                    clusters.ctypes.data, clusters.size, ctypes.byref(n_cl),
                                    triggers.ctypes.data, triggers.size, ctypes.byref(n_tr))
        return rc, n_cl.value, n_tr.value

    # -- the same path in three calls (global memory, no range size limit) --
    def tpx_decode(self, packets, hits_capacity: int | None = None, trig_capacity: int | None = None,
                   index_base: int = 0, n_packets: int | None = None) -> dict:
        """Kept pixels in stream order (device tensors) and the trigger times."""
        import torch
        n = int(packets.numel() if n_packets is None else n_packets)
        dev = torch.device("cuda", torch.cuda.current_device())
        cap = int(hits_capacity if hits_capacity is not None else max(1, n))
        tcap = int(trig_capacity if trig_capacity is not None else max(16, n))
        h = dict(index=torch.empty(cap, dtype=torch.int64, device=dev),
                 shot=torch.empty(cap, dtype=torch.int64, device=dev),
                 t=torch.empty(cap, dtype=torch.int64, device=dev),
                 tof=torch.empty(cap, dtype=torch.int32, device=dev),
                 x=torch.empty(cap, dtype=torch.uint8, device=dev),
                 y=torch.empty(cap, dtype=torch.uint8, device=dev),
                 tot=torch.empty(cap, dtype=torch.int16, device=dev))
        n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
        trig = torch.empty(tcap, dtype=torch.int64, device=dev)
        n_trig = torch.zeros(1, dtype=torch.int64, device=dev)
        ch = _CHits(*(_ptr(h[f]) for f in ("index", "shot", "t", "tof", "x", "y", "tot")))
        rc = lib().tpx_decode(self._h, _ptr(packets), n, int(index_base), ctypes.byref(ch), cap, _ptr(n_hits),
                              _ptr(trig), tcap, _ptr(n_trig))
        if rc:
            raise TpxError(rc, "tpx_decode")
        return dict(hits=h, n_hits=n_hits, trig=trig, n_trig=n_trig, hits_capacity=cap, trig_capacity=tcap)

    @staticmethod
    def _chits(h: dict) -> _CHits:
        return _CHits(*(_ptr(h[f]) for f in ("index", "shot", "t", "tof", "x", "y", "tot")))

    def tpx_tot_tof_histogram(self, hits: dict, n_hits: int, tof_lo_ticks: int, tof_bin_ticks: int,
                              n_tof_bins: int, hist=None):
        """Adds the ToT-ToF histogram of the hits' ToF window to `hist` (a zeroed
        device uint32 tensor of 1024 x n_tof_bins if None); returns it."""
        import torch
        if hist is None:
            hist = torch.zeros(1024 * n_tof_bins, dtype=torch.int32, device=hits["tof"].device)
        ch = self._chits(hits)
        rc = lib().tpx_tot_tof_histogram(self._h, ctypes.byref(ch), int(n_hits), int(tof_lo_ticks), int(tof_bin_ticks),
                                         int(n_tof_bins), _ptr(hist))
        if rc:
            raise TpxError(rc, "tpx_tot_tof_histogram")
        return hist

    def tpx_debug_hold_tile(self, tile: int):
        """The next tpx_process call holds tile `tile`'s look-back flags back
        (tests of the bounded device waits: tpx_sync then returns EDEVTIMEOUT)."""
        rc = lib().tpx_debug_hold_tile(self._h, int(tile))
        if rc:
            raise TpxError(rc, "tpx_debug_hold_tile")

    # -- the learned overlap refiner --
    def tpx_refine_patches(self, packets, labels, clusters, n_clusters: int, min_pixels: int = 12,
                           capacity: int | None = None, index_base: int = 0) -> dict:
        """Patches of the clusters with more than `min_pixels` pixels (device
        tensors: patches [n x 162] f32, sel [n] record index, centre [n x 2];
        n the number of such clusters, status 0 or TPX_EOVERFLOW)."""
        import torch
        dev = packets.device
        cap = int(capacity if capacity is not None else max(1, n_clusters))
        out = dict(patches=torch.empty((cap, 162), dtype=torch.float32, device=dev),
                   sel=torch.empty(cap, dtype=torch.int64, device=dev),
                   centre=torch.empty((cap, 2), dtype=torch.int32, device=dev),
                   n=torch.zeros(1, dtype=torch.int64, device=dev), capacity=cap)
        rc = lib().tpx_refine_patches(self._h, _ptr(packets), int(packets.numel()), int(index_base), _ptr(labels),
                                      _ptr(clusters), int(n_clusters), int(min_pixels), _ptr(out["patches"]),
                                      _ptr(out["sel"]), _ptr(out["centre"]), cap, _ptr(out["n"]))
        if rc and rc != EOVERFLOW:
            raise TpxError(rc, "tpx_refine_patches")
        out["status"] = rc   # TPX_EOVERFLOW: only the first `capacity` patches were written
        return out

    def tpx_refine_patches_bf16(self, packets, labels, clusters, n_clusters: int, min_pixels: int = 12,
                                capacity: int | None = None, index_base: int = 0) -> dict:
        """tpx_refine_patches with the patches as bf16 (device int16 tensor
        [n x 162] holding the bf16 bits)."""
        import torch
        dev = packets.device
        cap = int(capacity if capacity is not None else max(1, n_clusters))
        out = dict(patches=torch.empty((cap, 162), dtype=torch.int16, device=dev),
                   sel=torch.empty(cap, dtype=torch.int64, device=dev),
                   centre=torch.empty((cap, 2), dtype=torch.int32, device=dev),
                   n=torch.zeros(1, dtype=torch.int64, device=dev), capacity=cap)
        rc = lib().tpx_refine_patches_bf16(self._h, _ptr(packets), int(packets.numel()), int(index_base), _ptr(labels),
                                           _ptr(clusters), int(n_clusters), int(min_pixels), _ptr(out["patches"]),
                                           _ptr(out["sel"]), _ptr(out["centre"]), cap, _ptr(out["n"]))
        if rc and rc != EOVERFLOW:
            raise TpxError(rc, "tpx_refine_patches_bf16")
        out["status"] = rc
        return out

    # -- the convolutional refiner --
    @staticmethod
    def tpx_cnn_params() -> int:
        return int(lib().tpx_cnn_params())

    def tpx_cnn_forward(self, params, x, n: int | None = None, work=None, out=None):
        import torch
        n = int(x.shape[0] if n is None else n)
        if work is None:
            work = torch.empty(max(1, int(lib().tpx_cnn_work_floats(n))), dtype=torch.float32, device=x.device)
        if out is None:
            out = torch.empty((max(1, n), 6), dtype=torch.float32, device=x.device)
        rc = lib().tpx_cnn_forward(self._h, _ptr(params), _ptr(x), n, _ptr(work), _ptr(out))
        if rc:
            raise TpxError(rc, "tpx_cnn_forward")
        return out

    def tpx_cnn_train_step(self, params, adam_m, adam_v, grad, step: int, x, y, lr: float, offset_weight: float,
                           work, loss, n: int | None = None):
        n = int(x.shape[0] if n is None else n)
        rc = lib().tpx_cnn_train_step(self._h, _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(grad), int(step),
                                      _ptr(x), _ptr(y), n, float(lr), float(offset_weight), _ptr(work), _ptr(loss))
        if rc:
            raise TpxError(rc, "tpx_cnn_train_step")

    def tpx_cnn_pack(self, params, packed=None):
        import torch
        nb = int(lib().tpx_cnn_packed_bytes())
        if packed is None:
            packed = torch.empty(nb + 256, dtype=torch.uint8, device=params.device)
        rc = lib().tpx_cnn_pack(self._h, _ptr(params), _ptr(packed))
        if rc:
            raise TpxError(rc, "tpx_cnn_pack")
        return packed

    def tpx_cnn_infer(self, packed, x, n: int | None = None, work=None, out=None):
        """The CNN on the tensor cores; x: bf16 patches (int16 tensor of the
        bits, [n x 162])."""
        import torch
        n = int(x.shape[0] if n is None else n)
        if work is None:
            work = torch.empty(max(16, int(lib().tpx_cnn_infer_work_bytes(n))), dtype=torch.uint8, device=x.device)
        if out is None:
            out = torch.empty((max(1, n), 6), dtype=torch.float32, device=x.device)
        rc = lib().tpx_cnn_infer(self._h, _ptr(packed), _ptr(x), n, _ptr(work), _ptr(out))
        if rc:
            raise TpxError(rc, "tpx_cnn_infer")
        return out

    @staticmethod
    def tpx_refiner_params(hidden: int) -> int:
        return int(lib().tpx_refiner_params(int(hidden)))

    def tpx_refiner_forward(self, params, hidden: int, x, n: int | None = None, work=None, out=None):
        import torch
        n = int(x.shape[0] if n is None else n)
        if work is None:
            work = torch.empty(max(1, 2 * n * hidden), dtype=torch.float32, device=x.device)
        if out is None:
            out = torch.empty((max(1, n), 6), dtype=torch.float32, device=x.device)
        rc = lib().tpx_refiner_forward(self._h, _ptr(params), int(hidden), _ptr(x), n, _ptr(work), _ptr(out))
        if rc:
            raise TpxError(rc, "tpx_refiner_forward")
        return out

    def tpx_refiner_train_step(self, params, adam_m, adam_v, grad, hidden: int, step: int, x, y, lr: float,
                               offset_weight: float, work, loss, n: int | None = None):
        n = int(x.shape[0] if n is None else n)
        rc = lib().tpx_refiner_train_step(self._h, _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(grad), int(hidden),
                                          int(step), _ptr(x), _ptr(y), n, float(lr), float(offset_weight),
                                          _ptr(work), _ptr(loss))
        if rc:
            raise TpxError(rc, "tpx_refiner_train_step")

    def tpx_refiner_pack(self, params, hidden: int, packed=None):
        """The bf16 inference copy of fp32 parameters (device uint8 tensor)."""
        import torch
        nb = int(lib().tpx_refiner_packed_bytes(int(hidden)))
        if nb <= 0:
            raise TpxError(EUNSUPPORTED, "tpx_refiner_packed_bytes")
        if packed is None:
            packed = torch.empty(nb, dtype=torch.uint8, device=params.device)
        rc = lib().tpx_refiner_pack(self._h, _ptr(params), int(hidden), _ptr(packed))
        if rc:
            raise TpxError(rc, "tpx_refiner_pack")
        return packed

    def tpx_refiner_infer(self, packed, hidden: int, x, n: int | None = None, out=None):
        import torch
        n = int(x.shape[0] if n is None else n)
        if out is None:
            out = torch.empty((max(1, n), 6), dtype=torch.float32, device=x.device)
        rc = lib().tpx_refiner_infer(self._h, _ptr(packed), int(hidden), _ptr(x), n, _ptr(out))
        if rc:
            raise TpxError(rc, "tpx_refiner_infer")
        return out

    def tpx_refine_decide(self, out, clusters, sel, centre, n: int, threshold: float, hits=None):
        import torch
        if hits is None:
            hits = torch.empty((max(1, n), 5), dtype=torch.float32, device=out.device)
        rc = lib().tpx_refine_decide(self._h, _ptr(out), _ptr(clusters), _ptr(sel), _ptr(centre), int(n),
                                     float(threshold), _ptr(hits))
        if rc:
            raise TpxError(rc, "tpx_refine_decide")
        return hits

    def tpx_cluster(self, hits: dict, n_hits: int, is_peak: bool = True) -> dict:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        labels = torch.empty(max(1, n_hits), dtype=torch.int64, device=dev)
        pk = torch.empty(max(1, n_hits), dtype=torch.uint8, device=dev) if is_peak else None
        ch = self._chits(hits)
        rc = lib().tpx_cluster(self._h, ctypes.byref(ch), int(n_hits), _ptr(labels), _ptr(pk))
        if rc:
            raise TpxError(rc, "tpx_cluster")
        return dict(labels=labels, is_peak=pk)

    def tpx_centroid(self, hits: dict, labels, is_peak, n_hits: int, cluster_capacity: int | None = None) -> dict:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        cap = int(cluster_capacity if cluster_capacity is not None else max(16, n_hits))
        cl = torch.empty(cap * CLUSTER_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        n_cl = torch.zeros(1, dtype=torch.int64, device=dev)
        ch = self._chits(hits)
        rc = lib().tpx_centroid(self._h, ctypes.byref(ch), _ptr(labels), _ptr(is_peak), int(n_hits), _ptr(cl), cap,
                                _ptr(n_cl))
        if rc:
            raise TpxError(rc, "tpx_centroid")
        return dict(clusters=cl, n_clusters=n_cl, cluster_capacity=cap)


class Stream:
    """tpx_stream: acquisition chunks in, records of closed shots out."""

    def __init__(self, cfg: Config | None = None, max_chunk_packets: int = 1 << 20, max_hold_packets: int = 1 << 20,
                 hold_triggers: int = 2, slots: int = 4, hbm_budget_bytes: int = 0, stream=None):
        import torch
        cfg = cfg or Config()
        c = _CConfig(cfg.rx, cfg.ry, cfg.dt_ticks, cfg.mode, cfg.tof_max_ticks, cfg.wrap_thr_pix_ticks,
                     cfg.wrap_thr_tdc_ticks, _ptr(cfg.timewalk_lut), int(cfg.strict), 0)
        sc = _CStreamConfig(c, int(max_chunk_packets), int(max_hold_packets), int(hold_triggers), int(slots),
                            int(hbm_budget_bytes))
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        rc = lib().tpx_stream_create(ctypes.byref(h), ctypes.byref(sc), ctypes.c_void_p(self.stream.cuda_stream))
        if rc:
            raise TpxError(rc, "tpx_stream_create")
        self._h = h
        self._keep = cfg
        self._chunks = {}   # ticket -> chunk: the library reads it until the ticket is polled

    def submit(self, chunk: np.ndarray) -> int:
        """Queue a chunk; returns the ticket at once (raises TpxError, EAGAIN
        when all slots await poll). The chunk is held until its poll."""
        chunk = np.ascontiguousarray(chunk, dtype=np.uint64)
        t = ctypes.c_uint64()
        rc = lib().tpx_stream_submit(self._h, chunk.ctypes.data if chunk.size else None, chunk.size, ctypes.byref(t))
        if rc:
            raise TpxError(rc, "tpx_stream_submit")
        self._chunks[t.value] = chunk
        return t.value

    def finish(self) -> int:
        t = ctypes.c_uint64()
        rc = lib().tpx_stream_finish(self._h, ctypes.byref(t))
        if rc:
            raise TpxError(rc, "tpx_stream_finish")
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1) -> dict:
        r = _CStreamResult()
        rc = lib().tpx_stream_poll(self._h, ticket, ctypes.byref(r), int(timeout_us))
        if rc != ETIMEOUT:
            self._chunks.pop(ticket, None)
        if rc:
            raise TpxError(rc, "tpx_stream_poll")
        n = r.n_clusters
        cl = np.zeros(0, CLUSTER_DTYPE)
        if n:
            buf = (ctypes.c_char * (n * CLUSTER_DTYPE.itemsize)).from_address(r.clusters)
            cl = np.frombuffer(bytes(buf), CLUSTER_DTYPE).copy()
        tr = np.zeros(0, np.int64)
        if r.n_shots:
            tr = np.array((ctypes.c_int64 * r.n_shots).from_address(r.trig_t), dtype=np.int64)
        return dict(ticket=r.ticket, status=r.status, first_shot=r.first_shot, n_shots=r.n_shots, triggers=tr,
                    clusters=cl, packets_processed=r.packets_processed, latency_us=r.latency_us)

    def snapshot(self) -> bytes:
        """The stream's carry as a host byte block (poll pending results first)."""
        n = int(lib().tpx_stream_snapshot_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        w = ctypes.c_int64()
        rc = lib().tpx_stream_snapshot(self._h, buf, n, ctypes.byref(w))
        if rc:
            raise TpxError(rc, "tpx_stream_snapshot")
        return buf.raw[: w.value]

    def restore(self, block: bytes):
        """Continue a checkpointed stream (this stream must not have started)."""
        rc = lib().tpx_stream_restore(self._h, block, len(block))
        if rc:
            raise TpxError(rc, "tpx_stream_restore")

    def close(self):
        if getattr(self, "_h", None):
            lib().tpx_stream_destroy(self._h)   # processes what is queued first
            self._h = None
        self._chunks = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

