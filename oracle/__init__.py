"""CPU oracle for the TPX3 clustering / centroiding path -- TEST INFRASTRUCTURE.

Only tests/, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may
import this package. It is a plain sequential C program (tpx_oracle.c) that
shares no code with the CUDA path; see that file's header for the steps and
the paper passages each follows (Sec. III, IV.A-C, V.A-C).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_CC = 0
MODE_PAPER = 1
# 20 s in 1.5625 ns ticks (Sec. IV.A threshold for both streams)
WRAP_THR_TICKS = 12_800_000_000
# 100 us in ticks (Sec. IV.B background cut)
TOF_MAX_TICKS = 64_000

CLUSTER_DTYPE = np.dtype([("label", "<i8"), ("shot", "<i8"), ("t0", "<i8"), ("s_tot", "<i8"),
                          ("s_x", "<i8"), ("s_y", "<i8"), ("s_t", "<i8"), ("n", "<i4"),
                          ("n_peaks", "<i4"), ("x", "<f8"), ("y", "<f8"), ("tof", "<f8")])
INFO_DTYPE = np.dtype([("type", "<i4"), ("x", "<i4"), ("y", "<i4"), ("tot", "<i4"),
                       ("t", "<i8"), ("shot", "<i8"), ("tof", "<i8")])
COUNTER_FIELDS = ("packets", "pixels", "tdcs", "corrupt", "dropped_pre_trigger",
                  "dropped_background", "kept", "clusters", "peaks")


class _Cfg(ctypes.Structure):
    _fields_ = [("rx", ctypes.c_int32), ("ry", ctypes.c_int32), ("dt_ticks", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("tof_max_ticks", ctypes.c_int64),
                ("wrap_thr_pix_ticks", ctypes.c_int64), ("wrap_thr_tdc_ticks", ctypes.c_int64),
                ("timewalk_lut", ctypes.c_void_p), ("strict", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("epoch0_pix", ctypes.c_int64), ("epoch0_tdc", ctypes.c_int64),
                ("have_prev_pix", ctypes.c_int32), ("have_prev_tdc", ctypes.c_int32),
                ("prev_pix_raw", ctypes.c_int64), ("prev_tdc_raw", ctypes.c_int64)]


class _Counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in COUNTER_FIELDS]


@dataclasses.dataclass
class Config:
    rx: int = 1
    ry: int = 1
    dt_ticks: int = 32
    mode: int = MODE_CC
    tof_max_ticks: int = TOF_MAX_TICKS
    wrap_thr_pix_ticks: int = WRAP_THR_TICKS
    wrap_thr_tdc_ticks: int = WRAP_THR_TICKS
    timewalk_lut: np.ndarray | None = None
    strict: bool = False
    epoch0_pix: int = 0      # wraps before the first pixel packet (slices of a longer stream)
    epoch0_tdc: int = 0
    prev_pix_raw: int | None = None   # raw value of the pixel packet before the slice
    prev_tdc_raw: int | None = None   # raw value of the TDC packet before the slice


def _build() -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build() -> str:
    """Compile the oracle (building the checker is not using it)."""
    return _build()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build())
            L.orc_run.restype = ctypes.c_int
            L.orc_run.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(_Counters)]
            L.orc_free.argtypes = [ctypes.c_void_p]
            _lib = L
    return _lib


def run(packets: np.ndarray, cfg: Config | None = None, idx_base: int = 0, want_info: bool = False) -> dict:
    """Run the oracle on a packet array. Returns status, clusters (structured
    array, ascending label), labels (int64 per packet, -1 = not a kept pixel),
    is_peak (uint8 per packet), triggers (int64 unwrapped ticks), counters and,
    optionally, a per-packet info array (type, x, y, tot, t, shot, tof)."""
    cfg = cfg or Config()
    pk = np.ascontiguousarray(packets, dtype=np.uint64)
    n = pk.size
    c = _Cfg(cfg.rx, cfg.ry, cfg.dt_ticks, cfg.mode, cfg.tof_max_ticks, cfg.wrap_thr_pix_ticks,
             cfg.wrap_thr_tdc_ticks, None, int(cfg.strict), 0, int(cfg.epoch0_pix), int(cfg.epoch0_tdc),
             int(cfg.prev_pix_raw is not None), int(cfg.prev_tdc_raw is not None),
             int(cfg.prev_pix_raw or 0), int(cfg.prev_tdc_raw or 0))
    lut = None
    if cfg.timewalk_lut is not None:
        lut = np.ascontiguousarray(cfg.timewalk_lut, dtype=np.int16)
        assert lut.size == 1024
        c.timewalk_lut = lut.ctypes.data
    labels = np.empty(n, np.int64)
    is_peak = np.empty(n, np.uint8)
    info = np.empty(n, INFO_DTYPE) if want_info else None
    pcl = ctypes.c_void_p()
    ncl = ctypes.c_int64()
    ptr = ctypes.c_void_p()
    ntr = ctypes.c_int64()
    cnt = _Counters()
    L = lib()
    st = L.orc_run(ctypes.byref(c), pk.ctypes.data if n else None, n, idx_base, labels.ctypes.data,
                   is_peak.ctypes.data, info.ctypes.data if info is not None else None,
                   ctypes.byref(pcl), ctypes.byref(ncl), ctypes.byref(ptr), ctypes.byref(ntr),
                   ctypes.byref(cnt))
    out = dict(status=int(st), labels=labels, is_peak=is_peak)
    if st == -1:  # invalid arguments: nothing was produced
        out.update(clusters=np.zeros(0, CLUSTER_DTYPE), triggers=np.zeros(0, np.int64), counters={})
        return out
    m = ncl.value
    buf = (ctypes.c_char * (m * CLUSTER_DTYPE.itemsize)).from_address(pcl.value) if m else b""
    out["clusters"] = np.frombuffer(bytes(buf), CLUSTER_DTYPE).copy() if m else np.zeros(0, CLUSTER_DTYPE)
    L.orc_free(pcl)
    k = ntr.value
    tb = (ctypes.c_int64 * k).from_address(ptr.value) if k else []
    out["triggers"] = np.array(tb, dtype=np.int64)
    L.orc_free(ptr)
    out["counters"] = {f: int(getattr(cnt, f)) for f in COUNTER_FIELDS}
    if info is not None:
        out["info"] = info
    return out
