"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/tpx.h declares; host-only calls work
without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2603_04942_gb300 as tpx
from paper_2603_04942_gb300 import build as tbuild

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tpx.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpx_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return tbuild.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tpx_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(tpx.EXPORTED_SYMBOLS) <= exported


def test_library_loads_and_host_calls(libpath):
    L = tpx.load(libpath)
    for s in _declared():
        assert hasattr(L, s)
    cfg = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(cfg))
    assert (cfg.rx, cfg.ry, cfg.dt_ticks, cfg.tof_max_ticks) == (1, 1, 32, 64000)
    assert cfg.wrap_thr_pix_ticks == 12_800_000_000
    assert L.tpx_strerror(-3).decode().startswith("output buffer")
    assert b"sm_103a" in L.tpx_version()
    # invalid arguments are rejected before any CUDA work
    assert L.tpx_process(None, None, 0, 0, None, None, None, 0, None, None, 0, None) == tpx.EINVAL
    assert L.tpx_sync(None, None) == tpx.EINVAL
    assert L.tpx_destroy(None) == tpx.EINVAL
    bad = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(bad))
    bad.rx = 9
    h = ctypes.c_void_p()
    assert L.tpx_create(ctypes.byref(h), ctypes.byref(bad), 10, None) == tpx.EINVAL


def test_phase_counters_and_flags_without_a_gpu(libpath):
    L = tpx.load(libpath)
    arr = (ctypes.c_uint64 * 32)(*([7] * 32))
    # the normal build has no phase counters: unsupported, zeros
    assert L.tpx_debug_phase_times(tpx.TILE_2048, arr, 0) == tpx.EUNSUPPORTED
    assert list(arr) == [0] * 32
    assert L.tpx_debug_phase_times(5, arr, 0) == tpx.EINVAL
    arr16 = (ctypes.c_uint64 * 16)(*([7] * 16))
    assert L.tpx_debug_cnn_phase_times(arr16, 0) == tpx.EUNSUPPORTED
    assert list(arr16) == [0] * 16
    assert L.tpx_debug_cnn_phase_times(None, 0) == tpx.EINVAL
    assert L.tpx_kernel_timing(None, 1) == tpx.EINVAL
    assert L.tpx_kernel_times(None, None, None, None) == tpx.EINVAL
    # the configuration accepts the two flags and nothing else
    assert tpx.Config(labels32=True, host_direct=True).flags() == tpx.FLAG_LABELS32 | tpx.FLAG_HOST_DIRECT
    assert tpx.Config(records64=True).flags() == tpx.FLAG_RECORDS64
    assert tpx.CLUSTER64_DTYPE.names == tpx.CLUSTER_DTYPE.names[:9]
    bad = tpx._CConfig()
    L.tpx_config_default(ctypes.byref(bad))
    bad.flags = 32
    h = ctypes.c_void_p()
    assert L.tpx_create(ctypes.byref(h), ctypes.byref(bad), 10, None) == tpx.EINVAL


def test_build_targets_sm103a_only():
    assert tbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_cluster_record_layout():
    assert tpx.CLUSTER_DTYPE.itemsize == 88
    src = open(HDR).read()
    assert "} tpx_record;        /* 88 bytes */" in src


def test_product_path_has_no_oracle_import():
    """The package never reaches the oracle or a CPU fallback."""
    pkg = os.path.dirname(tpx.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "tpx_oracle" not in txt, f


def test_refiner_and_stream_host_calls(libpath):
    """Host-only entry points of the later additions: sizes and argument checks."""
    L = tpx.load(libpath)
    # 162 -> 160 -> 160 -> 6 with biases: 52,806 parameters; bf16 packing for 64/128/160 only
    assert L.tpx_refiner_params(160) == 162 * 160 + 160 + 160 * 160 + 160 + 160 * 6 + 6 == 52806
    assert L.tpx_refiner_params(0) == 0
    assert L.tpx_refiner_packed_bytes(160) > 0 and L.tpx_refiner_packed_bytes(128) > 0
    assert L.tpx_refiner_packed_bytes(100) == 0
    assert L.tpx_refiner_pack(None, None, 160, None) == tpx.EINVAL
    assert L.tpx_refiner_infer(None, None, 160, None, 0, None) == tpx.EINVAL
    assert L.tpx_refine_decide(None, None, None, None, None, 0, ctypes.c_float(0.5), None) == tpx.EINVAL
    assert L.tpx_debug_hold_tile(None, 3) == tpx.EINVAL
    assert L.tpx_stream_snapshot_bytes(None) == 0
    w = ctypes.c_int64()
    assert L.tpx_stream_snapshot(None, None, 0, ctypes.byref(w)) == tpx.EINVAL
    assert L.tpx_stream_restore(None, None, 0) == tpx.EINVAL
